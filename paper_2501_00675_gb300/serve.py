"""Continuous-batching evaluation server on one GPU.

Requests are (resident graph, number of samples, sample seed).  The server keeps
the graph structures resident (created once; every in-flight request on a graph
uses its own handle from ``cos_graph_share``, so several requests on one graph
run at once), admits requests in arrival order while their device memory fits a
budget, and keeps several persistent batched launches (``cos_batch_*``) in
flight on separate streams: requests that arrive while others run are admitted
as memory frees up and go into the next launch, whose work items start on the SMs
as the running launch drains.  Latency is measured from submission to the moment
the launch that carried the request is seen complete.

The evaluation itself runs in the CUDA library; this module only schedules.
``AdmissionController`` holds the host-side policy and has no GPU dependency.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Deque, Dict, List, Optional, Sequence, Tuple

import numpy as np


# ---------------------------------------------------------------------------- policy (no GPU)

@dataclasses.dataclass
class RequestSpec:
    graph_id: int
    num_samples: int
    seed: int


@dataclasses.dataclass
class Request:
    spec: RequestSpec
    need_bytes: int
    t_submit: float
    rid: int
    t_admit: float = 0.0
    t_launch: float = 0.0
    t_done: float = 0.0
    status: str = "queued"        # queued | admitted | running | done | shed | failed
    charged: int = 0
    mean: float = float("nan")
    result = None                 # device tensor of per-sample values
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class AdmissionController:
    """FIFO admission under a device-memory budget with a bounded wait queue.

    offer():   enqueue, or shed at once when the queue is full or the request can
               never fit the budget.
    admit():   pop queued requests in arrival order while their memory fits what is
               left of the budget (head-of-line: a request that does not fit yet
               blocks the ones behind it, so large requests are not starved).
               `cost(r)` gives the bytes admitting r charges now (default
               r.need_bytes), `can_run(r)` vetoes a request that lacks another
               resource, and `reclaim(n)` may free up to n bytes of idle memory
               (returns what it freed) before the head is refused; `on_admit(r)`
               runs right after r is admitted (e.g. to take the resources that
               `cost` and `can_run` looked at).
    release(): return bytes (default: the request's own charge).
    """

    def __init__(self, budget_bytes: int, max_queue: int = 1024):
        self.budget = int(budget_bytes)
        self.max_queue = int(max_queue)
        self.in_use = 0
        self.peak = 0
        self.queue: Deque[Request] = collections.deque()
        self.shed = 0
        self.admitted = 0

    def offer(self, req: Request) -> bool:
        if req.need_bytes > self.budget or len(self.queue) >= self.max_queue:
            req.status = "shed"
            self.shed += 1
            return False
        self.queue.append(req)
        return True

    def admit(self, max_n: int, cost=None, can_run=None, reclaim=None, on_admit=None) -> List[Request]:
        out = []
        while self.queue and len(out) < max_n:
            r = self.queue[0]
            if can_run is not None and not can_run(r):
                break
            need = r.need_bytes if cost is None else cost(r)
            if self.in_use + need > self.budget and reclaim is not None:
                self.in_use -= reclaim(self.in_use + need - self.budget)
            if self.in_use + need > self.budget:
                break
            self.queue.popleft()
            self.in_use += need
            self.peak = max(self.peak, self.in_use)
            r.charged = need
            r.status = "admitted"
            if on_admit is not None:
                on_admit(r)
            out.append(r)
        self.admitted += len(out)
        return out

    def release(self, req: Optional[Request] = None, nbytes: Optional[int] = None):
        self.in_use -= int(nbytes if nbytes is not None else req.need_bytes)
        assert self.in_use >= 0


def latency_summary(reqs: Sequence[Request]) -> Dict[str, float]:
    lat = np.array([r.latency for r in reqs if r.status == "done"])
    if lat.size == 0:
        return {"completed": 0}
    return {"completed": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "max_ms": float(lat.max() * 1e3)}


# ---------------------------------------------------------------------------- GPU server

def request_times(torch, spec: RequestSpec, num_times: int, beta: float):
    """Synthetic sample times of a request, drawn on the device from its seed: a
    [D][S_pad] buffer (S_pad = S rounded up to 128) of U[0, beta) values."""
    s_pad = max(128, (spec.num_samples + 127) // 128 * 128)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(int(spec.seed))
    return torch.rand((num_times, s_pad), generator=gen, device="cuda", dtype=torch.float64) * beta


class Server:
    """See the module docstring.

    graphs:       resident graphs, list of (binding.Graph, eps[K]) -- the pool
    mode:         evaluation mode of every request
    budget_bytes: device memory that admitted requests may hold at once
    max_batch:    requests per launch
    streams:      launches kept in flight
    tile_samples: tile of samples per request (bounds each request's workspace)
    single:       one request per launch through cos_evaluate (the plain path)
    """

    def __init__(self, graphs, mode: int, budget_bytes: int = 150 << 30, max_batch: int = 64, streams: int = 2,
                 tile_samples: int = 8192, max_queue: int = 4096, single: bool = False, beta: float = 10.0,
                 workspace_bytes: int = 512 << 20, handles_per_graph: int = 2):
        import torch
        from . import binding as cg
        self.torch = torch
        self.cg = cg
        self.graphs = [g for g, _ in graphs]
        self.eps = [np.ascontiguousarray(e, dtype=np.float64) for _, e in graphs]
        self.info = [g.info() for g in self.graphs]
        self.mode = mode
        self.beta = beta
        self.single = single
        self.max_batch = 1 if single else max_batch
        self.tile = tile_samples
        self.ws_bytes = workspace_bytes
        self.handles_per_graph = handles_per_graph
        self.ctrl = AdmissionController(budget_bytes, max_queue)
        # per graph: idle handles (cos_graph_share), and how many are in use; idle handles
        # keep their workspace charged to the budget until they are evicted (LRU)
        self.views: Dict[int, List] = collections.defaultdict(list)
        self.busy: Dict[int, int] = collections.defaultdict(int)
        self.idle_lru: "collections.OrderedDict" = collections.OrderedDict()
        self.evicted = 0
        self.n_streams = 1 if single else streams
        self.slots = []
        for _ in range(self.n_streams):
            st = torch.cuda.Stream()
            self.slots.append({"stream": st, "batch": None, "event": None, "reqs": None})
        self.requests: List[Request] = []
        self._lock = threading.Lock()
        self._inbox: Deque[Request] = collections.deque()
        self._rid = 0
        self.units_done = 0.0

    # -- memory model: workspace of one tile + the request's times and results
    def tile_for(self, graph_id: int) -> int:
        inf = self.info[graph_id]
        psb = 2 * 8 * inf["W_max"] + 8 * inf["P"]
        t = max(128, min(self.tile, (self.ws_bytes // psb) // 128 * 128))
        return int(t)

    def handle_bytes(self, graph_id: int) -> int:
        """Device memory of one evaluation handle of a graph: workspace of one tile of samples
        (sized for the double-precision layout) and small buffers."""
        inf = self.info[graph_id]
        psb = 2 * 8 * inf["W_max"] + 8 * inf["P"]
        return int(psb * ((self.tile_for(graph_id) + 127) // 128 * 128) + (8 << 20) + (1 << 20))

    def io_bytes(self, graph_id: int, num_samples: int) -> int:
        """Device memory of a request's own times [D][S_pad] and results [S]."""
        s_pad = max(128, (num_samples + 127) // 128 * 128)
        return int(s_pad * self.info[graph_id]["D"] * 8 + 8 * max(num_samples, 1))

    def need_bytes(self, graph_id: int, num_samples: int) -> int:
        """Upper bound of what admitting a request can charge (a new handle + its buffers)."""
        return self.handle_bytes(graph_id) + self.io_bytes(graph_id, num_samples)

    # -- admission callbacks
    def _cost(self, r: Request) -> int:
        g = r.spec.graph_id
        return self.io_bytes(g, r.spec.num_samples) + (0 if self.views[g] else self.handle_bytes(g))

    def _can_run(self, r: Request) -> bool:
        g = r.spec.graph_id
        return bool(self.views[g]) or self.busy[g] < self.handles_per_graph

    def _reclaim(self, nbytes: int) -> int:
        """Destroy least recently used idle handles until nbytes are freed."""
        freed = 0
        while freed < nbytes and self.idle_lru:
            (g, vid), v = self.idle_lru.popitem(last=False)
            self.views[g].remove(v)
            v.close()
            freed += self.handle_bytes(g)
            self.evicted += 1
        return freed

    def submit(self, spec: RequestSpec) -> Request:
        with self._lock:
            self._rid += 1
            req = Request(spec, self.need_bytes(spec.graph_id, spec.num_samples), time.perf_counter(), self._rid)
            self._inbox.append(req)
            self.requests.append(req)
        return req

    def _take_view(self, r: Request):
        r._view = self._view(r.spec.graph_id)

    def _view(self, gid: int):
        self.busy[gid] += 1
        pool = self.views[gid]
        if pool:
            v = pool.pop()
            self.idle_lru.pop((gid, id(v)), None)
            return v
        v = self.graphs[gid].share()
        v.set_tuning(tile_samples=self.tile_for(gid))
        return v

    def _return_view(self, gid: int, v):
        self.busy[gid] -= 1
        self.views[gid].append(v)
        self.idle_lru[(gid, id(v))] = v

    def _launch(self, slot, reqs: List[Request]):
        torch, cg = self.torch, self.cg
        st = slot["stream"]
        views, outs = [], []
        with torch.cuda.stream(st):
            for r in reqs:
                g = self.graphs[r.spec.graph_id]
                D = self.info[r.spec.graph_id]["D"]
                t = request_times(torch, r.spec, D, self.beta)
                v = r._view
                v.set_samples(t, self.eps[r.spec.graph_id], self.beta, cg.COS_T_BORROW,
                              num_samples=r.spec.num_samples, stream=st)
                dt = torch.int64 if self.mode == cg.COS_MODE_COUNT_I64 else torch.float64
                out = torch.empty(max(r.spec.num_samples, 1), dtype=dt, device="cuda")
                r.result = out[:r.spec.num_samples]
                r._t = t
                r._view = v
                views.append(v)
                outs.append(out)
                r.t_launch = time.perf_counter()
                r.status = "running"
            if self.single:
                views[0].evaluate(self.mode, out=outs[0], want_mean=False, stream=st)
            else:
                if slot["batch"] is None:
                    slot["batch"] = cg.Batch(views, self.mode, outs)
                else:
                    slot["batch"].reset(views, outs)
                slot["batch"].launch(stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        slot["event"] = ev
        slot["reqs"] = reqs

    def _finish(self, slot):
        reqs = slot["reqs"]
        now = time.perf_counter()
        try:
            if self.single:
                means = [reqs[0]._view.get_result(stream=slot["stream"])]
            else:
                means = slot["batch"].results(stream=slot["stream"])
            for r, m in zip(reqs, means):
                r.mean = float(m)
                r.status = "done"
        except Exception as exc:  # kernel-side error: report on every request of the launch
            for r in reqs:
                r.status = "failed"
                r.error = str(exc)
        for r in reqs:
            r.t_done = now
            self._return_view(r.spec.graph_id, r._view)   # its workspace stays charged while idle
            r._view = None
            r._t = None
            self.ctrl.release(nbytes=self.io_bytes(r.spec.graph_id, r.spec.num_samples))
            if r.status == "done":
                self.units_done += float(self.info[r.spec.graph_id]["E"]) * r.spec.num_samples
        slot["event"] = None
        slot["reqs"] = None

    def step(self) -> bool:
        """One scheduling pass; returns True if anything is queued or in flight."""
        with self._lock:
            while self._inbox:
                self.ctrl.offer(self._inbox.popleft())
        for slot in self.slots:
            if slot["event"] is not None and slot["event"].query():
                self._finish(slot)
        for slot in self.slots:
            if slot["event"] is None:
                reqs = self.ctrl.admit(self.max_batch, cost=self._cost, can_run=self._can_run,
                                       reclaim=self._reclaim, on_admit=self._take_view)
                if not reqs:
                    break
                now = time.perf_counter()
                for r in reqs:
                    r.t_admit = now
                self._launch(slot, reqs)
        busy = any(s["event"] is not None for s in self.slots)
        return busy or bool(self.ctrl.queue) or bool(self._inbox)

    def drain(self, timeout_s: float = 600.0):
        t0 = time.perf_counter()
        while self.step():
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(0.0002)

    def close(self):
        for slot in self.slots:
            if slot["event"] is not None:
                slot["event"].synchronize()
                self._finish(slot)
            if slot["batch"] is not None:
                slot["batch"].close()
        for pool in self.views.values():
            for v in pool:
                v.close()
        self.views.clear()
        self.idle_lru.clear()


class ResidentScheduler:
    """Continuous batching on the resident server (cos_server_*): one persistent
    kernel stays on the GPU and a request is handed to it as soon as a handle of its
    graph is free, so its work items start behind those already queued instead of
    at the next launch.  The kernel draws every request's sample times from the
    request's seed (counter-based generator), so admitting a request runs no kernel.

    Device memory is taken once, at construction: per graph one handle (workspace
    of one tile, time buffer and result buffer of max_samples), then a second
    handle per graph, smallest graphs first, while the budget lasts.  A request's
    per-sample values stay in its handle's result buffer until the handle's next
    request.  Same submit/step/drain/close interface as ``Server``.

    Order under load: the kernel's feeder shares the GPU round-robin among the
    requests it holds, so every request it holds slows the others down.  Requests
    are therefore handed to it oldest first and only while the work it holds (edges
    x samples of the requests not yet complete) stays within ``max_inflight_work``
    and their number within ``max_inflight`` -- enough to keep the GPU busy, few
    enough that a request admitted now finishes soon, whatever its size.  A request
    larger than the cap runs when it is the oldest and the GPU holds nothing else of
    the cap.  Younger requests never overtake an older one that waits for the cap
    (they may overtake one that waits for a handle of its graph).
    """

    def __init__(self, graphs, mode: int, budget_bytes: int = 150 << 30, max_samples: int = 1_000_000,
                 handles_per_graph: int = 2, tile_samples: int = 8192, workspace_bytes: int = 512 << 20,
                 max_queue: int = 4096, beta: float = 10.0, queue_tasks: int = 1 << 20, max_requests: int = 512,
                 idle_ms: int = 50, max_inflight: int = 64, max_inflight_work: float = 8e12):
        import torch
        from . import binding as cg
        self.torch, self.cg = torch, cg
        self.graphs = [g for g, _ in graphs]
        self.eps = [np.ascontiguousarray(e, dtype=np.float64) for _, e in graphs]
        self.info = [g.info() for g in self.graphs]
        self.mode, self.beta, self.tile, self.ws_bytes = mode, beta, tile_samples, workspace_bytes
        self.max_samples = int(max_samples)
        self.max_queue = int(max_queue)
        D = max(i["D"] for i in self.info)
        self.srv = cg.ResidentServer(mode, D, max_requests=max_requests, queue_tasks=queue_tasks, idle_ms=idle_ms)
        self.free: Dict[int, List] = collections.defaultdict(list)
        self.handles = []
        self.reserved = 0
        dt = torch.int64 if mode == cg.COS_MODE_COUNT_I64 else torch.float64
        order = sorted(range(len(self.graphs)), key=self.handle_bytes)
        for rnd in range(max(1, handles_per_graph)):
            for gid in order:
                need = self.handle_bytes(gid)
                if rnd > 0 and self.reserved + need > budget_bytes:
                    break
                h = self.graphs[gid].share()
                h.set_tuning(tile_samples=self.tile_for(gid))
                h.set_samples_uniform(self.max_samples, 0, self.eps[gid], beta)
                out = torch.empty(self.max_samples, dtype=dt, device="cuda")
                self.free[gid].append((h, out))
                self.handles.append(h)
                self.reserved += need
        torch.cuda.synchronize()
        self.queue: Deque[Request] = collections.deque()
        self.inflight: List[Request] = []
        self.requests: List[Request] = []
        self._lock = threading.Lock()
        self._inbox: Deque[Request] = collections.deque()
        self._rid = 0
        self.shed = 0
        self.units_done = 0.0
        self.max_inflight = int(max_inflight)
        self.max_inflight_work = float(max_inflight_work)

    def work_of(self, r) -> float:
        """Edges x samples of a request (its share of the GPU)."""
        return float(self.info[r.spec.graph_id]["E"]) * r.spec.num_samples

    def tile_for(self, graph_id: int) -> int:
        inf = self.info[graph_id]
        psb = 2 * 8 * inf["W_max"] + 8 * inf["P"]
        return int(max(128, min(self.tile, (self.ws_bytes // psb) // 128 * 128)))

    def handle_bytes(self, graph_id: int) -> int:
        """Workspace of one tile, times [D][max_samples] and results [max_samples]."""
        inf = self.info[graph_id]
        psb = 2 * 8 * inf["W_max"] + 8 * inf["P"]
        s_pad = (self.max_samples + 127) // 128 * 128
        return int(psb * self.tile_for(graph_id) + (8 << 20) + s_pad * 8 * (inf["D"] + 1))

    def submit(self, spec: RequestSpec) -> Request:
        with self._lock:
            self._rid += 1
            req = Request(spec, 0, time.perf_counter(), self._rid)
            self._inbox.append(req)
            self.requests.append(req)
        return req

    def step(self) -> bool:
        """One scheduling pass; returns True if anything is queued or in flight."""
        with self._lock:
            while self._inbox:
                r = self._inbox.popleft()
                if len(self.queue) >= self.max_queue or r.spec.num_samples > self.max_samples:
                    r.status = "shed"
                    self.shed += 1
                else:
                    self.queue.append(r)
        now = time.perf_counter()
        still = []
        for r in self.inflight:
            try:
                m = self.srv.poll(r._sid, allow_overflow=True)
            except self.cg.CosError as exc:
                r.status, r.error, m = "failed", str(exc), 0.0
            if m is None:
                still.append(r)
                continue
            r.t_done = now
            if r.status != "failed":
                r.status, r.mean = "done", float(m)
                self.units_done += float(self.info[r.spec.graph_id]["E"]) * r.spec.num_samples
            self.free[r.spec.graph_id].append(r._slot)
            r._slot = None
        self.inflight = still
        # admission: oldest first, while the held work and count stay within the caps
        # (the first request always fits); a request whose graph has no free handle
        # waits without holding up requests on other graphs
        cap_n = getattr(self, "max_inflight", 1 << 30)
        cap_w = getattr(self, "max_inflight_work", float("inf"))
        held = sum(self.work_of(r) for r in self.inflight)
        waiting = collections.deque()
        while self.queue:
            r = self.queue.popleft()
            if self.inflight and (len(self.inflight) >= cap_n or held + self.work_of(r) > cap_w):
                waiting.append(r)              # the caps are full: this one and every younger one wait
                waiting.extend(self.queue)
                self.queue.clear()
                break
            hl = self.free[r.spec.graph_id]
            if not hl:
                waiting.append(r)
                continue
            h, out = hl[-1]
            sid = self.srv.submit(h, r.spec.num_samples, r.spec.seed, out)
            if sid is None:   # no request slot or queue space: try again next pass
                waiting.append(r)
                waiting.extend(self.queue)
                self.queue.clear()
                break
            hl.pop()
            r._sid, r._slot = sid, (h, out)
            r.t_admit = r.t_launch = time.perf_counter()
            r.status = "running"
            self.inflight.append(r)
            held += self.work_of(r)
        self.queue = waiting
        return bool(self.inflight) or bool(self.queue) or bool(self._inbox)

    def drain(self, timeout_s: float = 600.0):
        t0 = time.perf_counter()
        while self.step():
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(0.0002)

    def close(self):
        self.drain()
        self.srv.close()
        for h in self.handles:
            h.close()
        self.handles = []
        self.free.clear()


def poisson_run(server: Server, specs: Sequence[RequestSpec], rate_per_s: float, duration_s: float,
                seed: int = 0) -> Tuple[List[Request], float]:
    """Submit specs at Poisson arrival times (rate_per_s) for at most duration_s while the
    scheduling loop runs in this thread; then drain.  Returns (requests, wall seconds)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=len(specs))
    arrivals = np.cumsum(gaps)
    t0 = time.perf_counter()
    k = 0
    while k < len(specs) and arrivals[k] <= duration_s:
        now = time.perf_counter() - t0
        while k < len(specs) and arrivals[k] <= now and arrivals[k] <= duration_s:
            server.submit(specs[k])
            k += 1
        server.step()
        time.sleep(0.0001)
    server.drain()
    return list(server.requests), time.perf_counter() - t0
