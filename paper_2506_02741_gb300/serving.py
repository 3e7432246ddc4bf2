"""Serving loops: many resident sections, render and track requests of uneven
resolution and size on one GPU.

* Sections (colour / opacity / radius in FP16 or FP32) stay resident on the
  device; a request names a section, a camera pose and a resolution bucket.
* ``render``: forward (colour, depth, silhouette); the colour image is copied
  to the host.  ``track``: one tracking iteration -- forward, the Eq. 1 masked
  L1 loss against the request's own observation (uploaded from the request's
  pinned host frame as part of the request) and the pose backward; the loss
  and the pose gradient are copied to the host.
* Latency runs from arrival to the result being visible on the host (a CUDA
  event after the device-to-host copy, polled without blocking).

BatchServer is the served form: continuous batching with one launch per
stage over all of a batch's items (vt_batch_*).  It keeps ``n_contexts`` batch contexts, each
with its own stream, workspace and capacity; whenever a context is idle it
takes queued requests (shortest estimated GPU time first, those waiting
longer than a limit first of all; or in arrival order) into one batch while
they fit its capacity (Gaussians, pixels, tiles, views, estimated tile
instances, 64 items) and their estimated GPU time stays within the batch's
budget -- a lone request goes at once, batches grow as requests queue up --
uploads their
poses and observations, launches the batch (replaying a CUDA graph captured
once per context) and copies the results back.  Requests that arrive while
batches run wait in the queue and are admitted as soon as a context frees
up; the contexts' batches overlap on the device.  The capacities come from
the free device memory at start-up (admission by free HBM): a request is
deferred until a context has room and refused only if it can never fit one.
A batch that exceeds the reserved tile instances on the device (found after
it ran) raises the estimates and is queued again.  A request admitted alone
(the queue held nothing else) runs on the context's single-request renderer
instead, replaying a graph captured per (section, bucket, kind): at low load
most requests go that way and skip the batched launches' work-item table.

SlotServer runs requests on ``n_slots`` independent render contexts (one
request per slot and stream), optionally replaying a CUDA graph per
(slot, section, bucket, kind); with one slot and no graphs it is the plain
one-request-at-a-time form.
"""

from __future__ import annotations

import collections
import contextlib
import dataclasses
import gc
import time

import numpy as np
import torch

from . import _lib as L
from . import api

TRACK_WEIGHTS = dict(w_rgb=0.5, w_depth=0.025, sil_min=0.99, rgb_needs_depth=True)


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "render" or "track"
    section: int
    pose: np.ndarray          # (3, 4) camera-to-world
    bucket: int               # index into the server's resolutions
    arrival: float = 0.0      # seconds from the start of the run
    obs: torch.Tensor | None = None   # track: pinned host (4, H, W) float32 (rgb, depth)
    done: float = -1.0
    result: torch.Tensor | None = None


def _pad(x: int) -> int:
    return (x + 255) // 256 * 256


def batch_budget(queued_ms, n_contexts: int, lo: float | None, hi: float) -> float:
    """GPU-time budget of the next batch: ``hi``, or with ``lo`` given the
    queued requests' estimated time divided among the contexts, clamped to
    [lo, hi]."""
    if lo is None:
        return hi
    return min(hi, max(lo, sum(queued_ms) / max(1, n_contexts)))


def admission_order(queue, now: float, ms_of, wait_ms: float) -> list:
    """The queue in admission order: requests that arrived more than wait_ms
    before ``now`` (seconds) first, oldest first; then the rest by estimated
    GPU time (ms_of), shortest first, ties by arrival."""
    late = now - wait_ms * 1e-3
    return sorted(queue, key=lambda q: (0, q.arrival, 0.0) if q.arrival < late else
                  (1, ms_of(q), q.arrival))


@contextlib.contextmanager
def _no_gc():
    """The serving loops hold Python's cyclic garbage collector off while they
    run (a collection pauses the loop for milliseconds, which shows up as
    latency of whatever request is due then); it runs once afterwards."""
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()
        gc.collect()


# ---------------------------------------------------------------------------
# Batched serving


class _BatchCtx:
    """One batch context: a BatchRunner with fixed pools for the items'
    images, observations, poses and results, and the pinned host buffers the
    results are copied to."""

    def __init__(self, server: "BatchServer", cap: dict):
        dev = server.device
        # one stream per priority level: a batch launched while k others run
        # goes on streams[k], so the GPU's block scheduler favours the
        # batches in the order they were admitted and a later batch fills
        # the SMs the earlier ones leave idle
        self.streams = [torch.cuda.Stream(device=dev, priority=-(server.n_contexts - 1 - k))
                        for k in range(server.n_contexts)]
        self.stream = self.streams[0]
        self.copy_stream = torch.cuda.Stream(device=dev)   # observation uploads
        self.cap = cap
        with torch.cuda.stream(self.stream):
            self.runner = api.BatchRunner(cap["gaussians"], cap["pixels"], cap["tiles"],
                                          cap["instances"], cap["views"], cap["table_rows"],
                                          list_cap=server.list_cap, stream=self.stream)
        P = cap["pixels"]
        n = self.max_items = 64      # VT_MAX_BATCH_ITEMS
        self.image = torch.empty(5 * P, device=dev)
        self.obs = torch.zeros(4 * P, device=dev)
        self.poses = torch.zeros(n, 12, dtype=torch.float64, device=dev)
        self.results = torch.zeros(n, 19, dtype=torch.float64, device=dev)
        self.poses_host = torch.zeros(n, 12, dtype=torch.float64).pin_memory()
        self.poses_np = self.poses_host.numpy()     # the same pinned memory
        self.results_host = torch.zeros(n, 19, dtype=torch.float64).pin_memory()
        self.rgb_host = torch.empty(3 * P, dtype=torch.float32).pin_memory()
        self.graph = None
        self.reqs: list[Request] = []
        self.slices: list[tuple] | None = []
        self.event = None
        self.mode = "batch"
        self.solo = None     # single-request renderer (_Slot), if the server keeps them
        self.work = None

    def busy(self) -> bool:
        return bool(self.reqs)


class BatchServer:
    def __init__(self, sections, resolutions, n_contexts: int = 2, graphs: bool = True,
                 memory_budget: int | None = None, list_cap: int = 256, batch_ms: float = 4.0,
                 graph_ms: float = 1.0, keep_results: bool = True, solo: bool = True,
                 batch_ms_min: float | None = 1.0, shortest_first_ms: float | None = 15.0,
                 device="cuda"):
        """sections: list of api.Section (resident, spheres); resolutions:
        list of (W, H) buckets.  The contexts share memory_budget (default:
        70% of the free device memory) in equal parts.  A batch takes queued
        requests while their estimated GPU time stays within its budget (the
        first request always goes), so that batches grow only when requests
        queue up.  The defaults are the policy measured best on the serving
        workload (two contexts, the budget following the queue between 1 and
        4 ms, shortest first within a 15 ms wait limit); batch_ms_min=None
        and shortest_first_ms=None give a fixed batch_ms budget and arrival
        order.  A batch whose estimated GPU time
        is below graph_ms replays the context's captured launch graph
        (persistent grids: launch overhead matters there); a longer one is
        launched directly with grids sized to its work, so that the stages of
        concurrent batches yield SMs block by block and the priority of the
        earlier batch holds.  With ``solo`` every context also keeps a
        single-request renderer with a captured graph per (section, bucket,
        kind): a request admitted alone runs there (the single-request
        kernels, no work-item table), a batch of two or more through the
        batched launches; the single-request renderers' memory counts against
        memory_budget.  With ``batch_ms_min`` the time budget of a batch
        follows the queue: its estimated GPU time divided among the contexts,
        clamped to [batch_ms_min, batch_ms].  With ``shortest_first_ms`` the
        queue is served shortest estimated GPU time first, except that the
        requests which have waited longer than that many milliseconds go
        first, oldest first (no request waits behind shorter ones for long)."""
        from . import synthetic as syn
        self.device = torch.device(device)
        self.sections = sections
        self.resolutions = [tuple(r) for r in resolutions]
        self.intrinsics = [syn.scaled_intrinsics(W, H).astuple() for W, H in self.resolutions]
        self.graphs = graphs
        self.list_cap = int(list_cap)
        self.batch_ms = float(batch_ms)
        self.batch_ms_min = None if batch_ms_min is None else float(batch_ms_min)
        self.shortest_first_ms = None if shortest_first_ms is None else float(shortest_first_ms)
        self.graph_ms = float(graph_ms)
        self.keep_results = keep_results
        free, _ = torch.cuda.mem_get_info(self.device)
        self._budget_arg = memory_budget
        self.memory_budget = int(memory_budget if memory_budget is not None else 0.7 * free)
        self.n_contexts = int(n_contexts)
        self.solo = bool(solo)
        self.solo_off: set = set()     # (section, bucket, kind) that overflowed a solo workspace
        self.n_solo = 0                # requests served alone / in batched launches
        self.n_batched = 0
        self.ctxs: list[_BatchCtx] = []
        # tile instances per (section, bucket): measured at warm-up, raised
        # when a batch overflows; GPU milliseconds per (section, bucket, kind)
        self.inst_est: dict = {}
        self.ms_est: dict = {}
        self.splits = 0

    # -- capacity -------------------------------------------------------------
    def _need(self, r: Request) -> dict:
        s = self.sections[r.section]
        W, H = self.resolutions[r.bucket]
        return dict(gaussians=_pad(s.n), pixels=_pad(W * H),
                    tiles=((W + 15) // 16) * ((H + 15) // 16), views=s.n_views,
                    table_rows=s.n_views * (s.depth.shape[-1] + s.depth.shape[-2]),
                    instances=int(self.inst_est.get((r.section, r.bucket), 6 * s.n + 65536)))

    def _ms(self, r: Request) -> float:
        k = (r.section, r.bucket, r.kind)
        if k in self.ms_est:
            return self.ms_est[k]
        return float(np.mean(list(self.ms_est.values()))) if self.ms_est else self.batch_ms

    def _bytes(self, cap) -> int:
        return api.BatchRunner.workspace_bytes_for(
            cap["gaussians"], cap["pixels"], cap["tiles"], cap["instances"], cap["views"],
            cap["table_rows"], self.list_cap) + 36 * cap["pixels"]

    def _capacity(self, requests) -> dict:
        """Per-context capacity: room for the largest request and for
        ``per_batch`` average requests (the batches batch_ms allows), within
        the context's share of the memory budget."""
        needs = [self._need(r) for r in requests]
        big = {k: max(n[k] for n in needs) for k in needs[0]}
        mean = {k: float(np.mean([n[k] for n in needs])) for k in needs[0]}
        ms = float(np.mean([self._ms(r) for r in requests]))
        per_batch = int(min(64, max(2, 2.0 * self.batch_ms / max(ms, 1e-3))))
        share = self.memory_budget // max(1, self.n_contexts)
        cap = {k: int(max(big[k], per_batch * mean[k])) for k in big}
        while self._bytes(cap) > share and any(cap[k] > big[k] for k in cap):
            cap = {k: int(max(big[k], 0.85 * cap[k])) for k in cap}
        if self._bytes(cap) > share:
            raise MemoryError(f"the largest request needs {self._bytes(cap)} bytes, more than "
                              f"a context's share {share} of the budget")
        return cap

    def _measure_instances(self, requests):
        """Tile instances of one render of every (section, bucket) the
        requests use, at one of their poses, with a 1.5x margin."""
        R = api.Renderer()
        seen = {}
        for r in requests:
            seen.setdefault((r.section, r.bucket), r)
        for (s, b), r in seen.items():
            W, H = self.resolutions[b]
            R.render([self.sections[s]], api.pose12(r.pose, self.device), self.intrinsics[b], W, H,
                     checked=True)
            self.inst_est[(s, b)] = int(1.5 * R.needed_instances()) + 4096
        del R
        torch.cuda.synchronize()

    def _measure_times(self, ctx, requests):
        """GPU time of a one-item batch of every (section, bucket, kind) the
        requests use, at the pose of the first such request (CUDA events,
        second of two runs)."""
        seen = {}
        for r in requests:
            seen.setdefault((r.section, r.bucket, r.kind), r)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for key, r in seen.items():
            r = dataclasses.replace(r, obs=self._dummy_obs(r))
            items, _ = self._items(ctx, [r])
            with torch.cuda.stream(ctx.stream):
                ctx.poses[0].copy_(api.pose12(r.pose, self.device))
                for _ in range(2):
                    if r.kind == "track":
                        items[0].obs.copy_(r.obs, non_blocking=True)
                    ctx.runner.set(self.sections, items, **TRACK_WEIGHTS)
                    e0.record(ctx.stream)
                    ctx.runner.launch(stream=ctx.stream)
                    e1.record(ctx.stream)
                e1.synchronize()
            ctx.runner.status(ctx.stream)
            self.ms_est[key] = e0.elapsed_time(e1)

    def warm(self, requests):
        """Measure instance counts, create the contexts, time every kind of
        request once, run one batch on each context and capture its launch
        graph.  Estimates and single-request graphs are made for every
        (section, bucket, kind), also those the given requests do not use (at
        a pose of a request of the same section, else of the first request),
        so that none is missing or captured while requests are served; the
        contexts' capacities follow the given requests."""
        every = self._cover(requests)
        self._measure_instances(every)
        probe = _BatchCtx(self, {k: v for k, v in self._need_max(every).items()})
        self._measure_times(probe, every)
        del probe
        torch.cuda.synchronize()
        solos = self._make_solos(every) if self.solo else [None] * self.n_contexts
        cap = self._capacity(requests)
        self.ctxs = [_BatchCtx(self, cap) for _ in range(self.n_contexts)]
        for ctx, slot in zip(self.ctxs, solos):
            ctx.solo = slot
        for ctx in self.ctxs:
            r = requests[0]
            self._launch(ctx, [dataclasses.replace(r, obs=self._dummy_obs(r))], warmup=True)
            ctx.event.synchronize()
            ctx.reqs = []
        torch.cuda.synchronize()

    def _make_solos(self, requests):
        """One single-request renderer per context, its workspace reserved for
        the largest request and a graph captured for every (section, bucket,
        kind) of ``requests``; the memory it takes leaves the contexts'
        budget (the default budget is taken from the free memory after)."""
        free0, _ = torch.cuda.mem_get_info(self.device)
        n_max = max(self.sections[r.section].n for r in requests)
        i_max = max(self._need(r)["instances"] for r in requests)
        seen = {}
        for r in requests:
            seen.setdefault((r.section, r.bucket, r.kind), r)
        solos = []
        for i in range(self.n_contexts):
            slot = _Slot(self, i)
            slot.reserve_for(self, n_max, i_max)
            for r in seen.values():
                slot.work_for(self, dataclasses.replace(r, obs=self._dummy_obs(r)), slot.stream,
                              self.graphs)
            solos.append(slot)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(self.device)
        if self._budget_arg is None:
            self.memory_budget = int(0.7 * free1)
        else:
            self.memory_budget = int(self._budget_arg) - max(0, free0 - free1)
        return solos

    def _cover(self, requests) -> list:
        seen = {(r.section, r.bucket, r.kind) for r in requests}
        pose_of = {}
        for r in requests:
            pose_of.setdefault(r.section, r.pose)
        extra = []
        for s in range(len(self.sections)):
            for b in range(len(self.resolutions)):
                for kind in ("render", "track"):
                    if (s, b, kind) not in seen:
                        extra.append(Request(-1, kind, s, pose_of.get(s, requests[0].pose), b))
        return list(requests) + extra

    def _need_max(self, requests) -> dict:
        needs = [self._need(r) for r in requests]
        return {k: max(n[k] for n in needs) for k in needs[0]}

    def _dummy_obs(self, r):
        if r.kind != "track":
            return None
        W, H = self.resolutions[r.bucket]
        return r.obs if r.obs is not None else torch.zeros(4, H, W).pin_memory()

    # -- batches -------------------------------------------------------------
    def _fits(self, ctx, used, need, ms, budget) -> bool:
        return (used["items"] < ctx.max_items and used["ms"] + ms <= budget and
                all(used[k] + need[k] <= ctx.cap[k] for k in ctx.cap))

    def _items(self, ctx, reqs):
        items, slices = [], []
        off = 0
        for i, r in enumerate(reqs):
            W, H = self.resolutions[r.bucket]
            P = W * H
            img = ctx.image[5 * off:5 * off + 5 * P].view(5, H, W)
            it = api.BatchItem(r.section, r.kind == "track", W, H, self.intrinsics[r.bucket],
                               ctx.poses[i], img)
            if r.kind == "track":
                it.obs = ctx.obs[4 * off:4 * off + 4 * P].view(4, H, W)
                it.result = ctx.results[i]
            items.append(it)
            slices.append((off, P, W, H))
            off += _pad(P)
        return items, slices

    def _launch(self, ctx, reqs, warmup=False, level=0):
        items, slices = self._items(ctx, reqs)
        ctx.stream = ctx.streams[min(level, len(ctx.streams) - 1)]
        with torch.cuda.stream(ctx.stream):
            n = len(reqs)
            p = np.stack([np.asarray(r.pose, np.float64).reshape(3, 4) for r in reqs])
            ctx.poses_np[:n, :9] = p[:, :, :3].reshape(n, 9)
            ctx.poses_np[:n, 9:] = p[:, :, 3]
            ctx.poses.copy_(ctx.poses_host, non_blocking=True)
            use_graph = (ctx.graph is not None and not warmup and
                         sum(self._ms(r) for r in reqs) < self.graph_ms)
            obs_ready = None
            if any(r.kind == "track" for r in reqs):
                # each track request's own observation: on the copy stream
                # while the render stages run (directly launched batches),
                # before the replay (captured ones)
                cs = ctx.stream if use_graph or warmup else ctx.copy_stream
                cs.wait_stream(ctx.stream)
                with torch.cuda.stream(cs):
                    for it, r in zip(items, reqs):
                        if r.kind == "track":
                            it.obs.copy_(r.obs, non_blocking=True)
                if cs is ctx.copy_stream:
                    obs_ready = torch.cuda.Event()
                    obs_ready.record(cs)
            ctx.runner.set(self.sections, items, **TRACK_WEIGHTS)
            if self.graphs and ctx.graph is None and warmup:
                ctx.runner.launch(stream=ctx.stream)      # eager once, then capture
                ctx.stream.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=ctx.stream):
                    ctx.runner.launch(stream=ctx.stream)
                ctx.graph = g
                ctx.runner.set(self.sections, items, **TRACK_WEIGHTS)
            if use_graph:
                ctx.graph.replay()
            else:
                ctx.runner.launch(stream=ctx.stream, obs_ready=obs_ready)
            n = len(reqs)
            if any(r.kind == "track" for r in reqs):
                ctx.results_host[:n].copy_(ctx.results[:n], non_blocking=True)
            for (off, P, W, H), r in zip(slices, reqs):
                if r.kind == "render":
                    ctx.rgb_host[3 * off:3 * off + 3 * P].copy_(ctx.image[5 * off:5 * off + 3 * P],
                                                                non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(ctx.stream)
        ctx.reqs, ctx.slices, ctx.event, ctx.mode = list(reqs), slices, ev, "batch"

    def _launch_solo(self, ctx, r, level=0):
        """A lone request on the context's single-request renderer (its
        graph for the request's section, bucket and kind), on the stream of
        the given priority level."""
        ctx.stream = ctx.streams[min(level, len(ctx.streams) - 1)]
        slot = ctx.solo
        work = slot.work_for(self, r, ctx.stream, self.graphs)
        with torch.cuda.stream(ctx.stream):
            slot.stage_pose(r.pose, work)
            if r.kind == "track":
                work.obs.copy_(r.obs, non_blocking=True)
            if work.graph is not None:
                work.graph.replay()
            else:
                work.run()
            work.host.copy_(work.rgb if r.kind == "render" else work.out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(ctx.stream)
        ctx.reqs, ctx.slices, ctx.event, ctx.mode, ctx.work = [r], None, ev, "solo", work

    def _finish(self, ctx, now, finished, queue):
        if ctx.mode == "solo":
            r = ctx.reqs[0]
            try:
                ctx.solo.renderer.status(ctx.stream)
            except L.VTError as e:
                if e.status != L.VT_ERR_CAPACITY:
                    raise
                # beyond the solo workspace: this kind goes through batches
                self.solo_off.add((r.section, r.bucket, r.kind))
                queue.appendleft(r)
                ctx.reqs = []
                return
            r.done = now
            if self.keep_results:
                r.result = ctx.work.host.clone()
            finished.append(r)
            self.n_solo += 1
            ctx.reqs = []
            return
        try:
            ctx.runner.status(ctx.stream)
        except L.VTError as e:
            if e.status != L.VT_ERR_CAPACITY:
                raise
            # more tile instances than estimated: raise the estimates of the
            # batch's (section, bucket) pairs and queue its requests again
            for r in ctx.reqs:
                k = (r.section, r.bucket)
                self.inst_est[k] = 2 * self.inst_est.get(k, 0) + 65536
            self.splits += 1
            for r in reversed(ctx.reqs):
                queue.appendleft(r)
            ctx.reqs = []
            return
        for i, ((off, P, W, H), r) in enumerate(zip(ctx.slices, ctx.reqs)):
            r.done = now
            if self.keep_results:
                if r.kind == "render":
                    r.result = ctx.rgb_host[3 * off:3 * off + 3 * P].view(3, H, W).clone()
                else:
                    r.result = ctx.results_host[i].clone()
            finished.append(r)
        self.n_batched += len(ctx.reqs)
        ctx.reqs = []

    def run(self, requests, timeout: float = 600.0):
        """Serve ``requests`` (arrival times in seconds from now).  Returns
        them with ``done`` (and ``result``) set."""
        with _no_gc():
            return self._run(requests, timeout)

    def _run(self, requests, timeout):
        for r in requests:
            n = self._need(r)
            if any(n[k] > self.ctxs[0].cap[k] for k in ("gaussians", "pixels", "tiles", "views",
                                                         "table_rows")):
                raise ValueError(f"request {r.rid} can never fit a batch context")
        queue = collections.deque()
        pending = list(sorted(requests, key=lambda r: r.arrival))
        nxt, finished = 0, []
        t0 = time.perf_counter()
        while len(finished) < len(requests):
            now = time.perf_counter() - t0
            if now > timeout:
                raise TimeoutError("serving run exceeded its time limit")
            while nxt < len(pending) and pending[nxt].arrival <= now:
                queue.append(pending[nxt])
                nxt += 1
            for ctx in self.ctxs:          # completions (non-blocking)
                if ctx.busy() and ctx.event.query():
                    self._finish(ctx, time.perf_counter() - t0, finished, queue)
            for ctx in self.ctxs:          # admissions in arrival order
                if ctx.busy() or not queue:
                    continue
                used = dict(gaussians=0, pixels=0, tiles=0, views=0, table_rows=0, instances=0,
                            items=0, ms=0.0)
                budget = batch_budget([self._ms(q) for q in queue], self.n_contexts,
                                      self.batch_ms_min, self.batch_ms)
                if self.shortest_first_ms is not None and len(queue) > 1:
                    queue = collections.deque(admission_order(queue, now, self._ms,
                                                              self.shortest_first_ms))
                take = [queue.popleft()]   # the head always goes (it fits an empty context)
                for k, v in self._need(take[0]).items():
                    used[k] += v
                used["items"], used["ms"] = 1, self._ms(take[0])
                while queue:
                    need, ms = self._need(queue[0]), self._ms(queue[0])
                    if not self._fits(ctx, used, need, ms, budget):
                        break
                    for k in need:
                        used[k] += need[k]
                    used["items"] += 1
                    used["ms"] += ms
                    take.append(queue.popleft())
                level = sum(c.busy() for c in self.ctxs)
                if (len(take) == 1 and ctx.solo is not None and
                        (take[0].section, take[0].bucket, take[0].kind) not in self.solo_off):
                    self._launch_solo(ctx, take[0], level)
                else:
                    self._launch(ctx, take, level=level)
            if all(c.busy() for c in self.ctxs) or (not queue and nxt < len(pending)):
                time.sleep(20e-6)
        return finished


# ---------------------------------------------------------------------------
# One request per slot


class _Work:
    """A captured graph (optional) for one (slot, section, bucket, kind); the
    buffers are the slot's for the (bucket, kind), shared by every section
    (a slot runs one request at a time)."""

    def __init__(self, slot, server, section, bucket, kind):
        W, H = server.resolutions[bucket]
        self.slot, self.kind, self.W, self.H = slot, kind, W, H
        self.K = server.intrinsics[bucket]
        self.sec = server.sections[section]
        b = slot.buffers(server.device, bucket, W, H, kind)
        self.pose, self.rgb, self.depth, self.sil = b["pose"], b["rgb"], b["depth"], b["sil"]
        self.d_twist, self.d_mat, self.loss = b["d_twist"], b["d_mat"], b["loss"]
        self.g_rgb, self.g_depth, self.obs = b["g_rgb"], b["g_depth"], b["obs"]
        self.out, self.host = b["out"], b["host"]
        self.graph = None

    def run(self):
        R = self.slot.renderer
        R.render([self.sec], self.pose, self.K, self.W, self.H, self.rgb, self.depth, self.sil)
        if self.kind == "track":   # Eq. 1 masked L1 (alpha 0.5, beta 0.025), pose gradient
            R.masked_l1(self.rgb, self.depth, self.sil, self.obs[:3], self.obs[3], 0.5, 0.025,
                        sil_min=0.99, rgb_needs_depth=True, d_rgb=self.g_rgb,
                        d_depth=self.g_depth, loss=self.loss)
            self.d_twist.zero_()
            self.d_mat.zero_()
            R.backward(self.g_rgb, self.g_depth, None, pose_grad=True, d_twist=self.d_twist,
                       d_mat=self.d_mat)
            # the batched form's result layout: loss, dL/dtwist, dL/d[R|t]
            self.out[:1].copy_(self.loss)
            self.out[1:7].copy_(self.d_twist)
            self.out[7:].copy_(self.d_mat)


class _Slot:
    def __init__(self, server, index):
        self.index = index
        self.stream = torch.cuda.Stream(device=server.device)
        self.renderer = api.Renderer()
        self.works = {}
        self.bufs = {}
        self.request = None
        self.event = None
        self.reserved = (0, 0, 0)    # Gaussians, pixels, instances
        self.work = None
        self.pose_host = torch.zeros(12, dtype=torch.float64).pin_memory()
        self.pose_np = self.pose_host.numpy()

    def buffers(self, dev, bucket, W, H, kind) -> dict:
        key = (bucket, kind)
        if key not in self.bufs:
            f = lambda *shape: torch.zeros(*shape, device=dev)
            d = lambda n: torch.zeros(n, dtype=torch.float64, device=dev)
            b = dict(pose=d(12), rgb=f(3, H, W), depth=f(H, W), sil=f(H, W))
            if kind == "track":
                b.update(d_twist=d(6), d_mat=d(12), loss=d(1), g_rgb=f(3, H, W),
                         g_depth=f(H, W), obs=f(4, H, W), out=d(19),
                         host=torch.empty(19, dtype=torch.float64).pin_memory())
            else:
                b.update(d_twist=None, d_mat=None, loss=None, g_rgb=None, g_depth=None,
                         obs=None, out=None, host=torch.empty(3, H, W).pin_memory())
            self.bufs[key] = b
        return self.bufs[key]

    def stage_pose(self, pose, work):
        """Copies a (3, 4) pose into the work's device pose buffer through the
        slot's pinned staging buffer (current stream)."""
        p = np.asarray(pose, np.float64).reshape(3, 4)
        self.pose_np[:9] = p[:, :3].reshape(9)
        self.pose_np[9:] = p[:, 3]
        work.pose.copy_(self.pose_host, non_blocking=True)

    def reserve_for(self, server, n_max, i_max):
        """Reserves the renderer's workspace for the largest request (captured
        graphs hold its addresses, so it must not move afterwards) and
        renders once at the largest size, which allocates the per-pixel
        lists."""
        b_max = max(range(len(server.resolutions)),
                    key=lambda b: server.resolutions[b][0] * server.resolutions[b][1])
        W, H = server.resolutions[b_max]
        with torch.cuda.stream(self.stream):
            self.renderer.reserve(n_max, W, H, i_max)
            work = _Work(self, server, max(range(len(server.sections)),
                                           key=lambda s: server.sections[s].n), b_max, "render")
            work.run()
        self.reserved = (n_max, W * H, i_max)

    def work_for(self, server, req, stream, graphs: bool):
        """The slot's work for the request's (section, bucket, kind), created
        (and its graph captured on ``stream``) on first use."""
        key = (req.section, req.bucket, req.kind)
        work = self.works.get(key)
        if work is None:
            work = _Work(self, server, req.section, req.bucket, req.kind)
            self.works[key] = work
            if graphs:
                with torch.cuda.stream(stream):
                    self.stage_pose(req.pose, work)
                    work.run()                      # warm-up outside the capture
                    stream.synchronize()
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=stream):
                        work.run()
                    work.graph = g
        return work


class SlotServer:
    def __init__(self, sections, resolutions, n_slots: int = 4, graphs: bool = True,
                 memory_budget: int | None = None, keep_results: bool = True, device="cuda"):
        """sections: list of api.Section (resident); resolutions: list of
        (W, H) buckets."""
        from . import synthetic as syn
        self.device = torch.device(device)
        self.sections = sections
        self.resolutions = [tuple(r) for r in resolutions]
        self.intrinsics = [syn.scaled_intrinsics(W, H).astuple() for W, H in self.resolutions]
        self.graphs = graphs
        self.keep_results = keep_results
        self.slots = [_Slot(self, i) for i in range(n_slots)]
        free, total = torch.cuda.mem_get_info(self.device)
        self.memory_budget = memory_budget if memory_budget is not None else int(free * 0.8)
        self.max_instances_per_gaussian = 6.0

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
        W, H = max(self.resolutions, key=lambda wh: wh[0] * wh[1])
        per_slot = api.L.lib().vt_workspace_bytes(n_max, W, H, i_max) + 8 * 256 * W * H
        usable = max(1, min(len(self.slots), self.memory_budget // max(per_slot, 1)))
        self.slots = self.slots[:usable]
        for slot in self.slots:
            slot.reserve_for(self, n_max, i_max)
        torch.cuda.synchronize()

    def _launch(self, slot, req):
        work = slot.work_for(self, req, slot.stream, self.graphs)
        with torch.cuda.stream(slot.stream):
            slot.stage_pose(req.pose, work)
            if req.kind == "track":           # the request's own observation
                work.obs.copy_(req.obs, non_blocking=True)
            if work.graph is not None:
                work.graph.replay()
            else:
                work.run()
            work.host.copy_(work.rgb if req.kind == "render" else work.out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.request, slot.event, slot.work = req, ev, work

    def warm(self, requests):
        """Size the slot workspaces and capture the graphs for every
        (slot, section, bucket, kind) the requests use."""
        self._size_slots(requests)
        seen = {}
        for r in requests:
            seen.setdefault((r.section, r.bucket, r.kind), r)
        for r in seen.values():
            for slot in self.slots:
                self._launch(slot, r)
                slot.event.synchronize()
                slot.request = None
        torch.cuda.synchronize()

    def run(self, requests, timeout: float = 600.0):
        """Serve ``requests`` (sorted by arrival time, in seconds from now).
        Returns the requests with ``done`` set and their results."""
        with _no_gc():
            return self._run(requests, timeout)

    def _run(self, requests, timeout):
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
                    if self.keep_results:
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
            "mpix_s": pix / span / 1e6, "req_s": len(done) / span, "span_s": span}


def poisson_requests(n, rate_per_s, n_sections, n_buckets, poses, seed=3, track_frac=0.7,
                     frames=None):
    """Seeded request stream: Poisson arrivals, 70% track / 30% render,
    uniform section and resolution; poses drawn from ``poses`` (per section);
    frames[b] (a list of pinned host (4, H, W) observations of bucket b), if
    given, supply the track requests' observations."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    out = []
    for i in range(n):
        kind = "track" if rng.random() < track_frac else "render"
        s = int(rng.integers(n_sections))
        b = int(rng.integers(n_buckets))
        pose = poses[s][int(rng.integers(len(poses[s])))]
        obs = None
        if kind == "track" and frames is not None:
            obs = frames[b][int(rng.integers(len(frames[b])))]
        out.append(Request(i, kind, s, pose, b, arrival=float(t[i]), obs=obs))
    return out
