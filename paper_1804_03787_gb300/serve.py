"""Serving: continuous batching over the C ABI with size-aware HBM admission.

Frame pairs of different sizes arrive over time.  A request is admitted when
the device state it needs fits the HBM budget: its frame size is rounded up to
a size class (multiples of ``size_quantum`` pixels per side), and a context of
that class -- a gpm context with its own CUDA stream, frame, flow and
occlusion buffers and pinned host staging -- costs gpm_required_bytes for the
class plus those buffers.  A finished request leaves its context idle in a
per-class cache, so the next request of the class starts without allocating;
when a new context does not fit, idle contexts of other classes are destroyed
(least recently used first).  A request that still does not fit is refused
with GPM_EBUSY and waits in arrival order (first come, first served: a later,
smaller request does not overtake it).  A cancelled request leaves the queue,
or, when it is already running, its result is dropped and its context is
freed as soon as its kernels finish.

Every request's result depends only on its frames, its pair id and the
parameters: the same alone and in any mix (tests/test_serve.py checks this).
"""
from __future__ import annotations

import ctypes as C
import math
import time
from dataclasses import dataclass

import numpy as np

from . import gpm


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds from the start of the trace
    frame1: np.ndarray             # float32 H x W x 3 (host)
    frame2: np.ndarray
    pair_id: int = 0
    t_start: float = -1.0
    t_done: float = -1.0
    flow: np.ndarray | None = None
    occ: np.ndarray | None = None
    cancelled: bool = False
    refusals: int = 0              # admissions refused with GPM_EBUSY while it waited at the head of the queue

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival

    @property
    def size(self) -> tuple[int, int]:
        return self.frame1.shape[1], self.frame1.shape[0]


def io_bytes(width: int, height: int) -> int:
    """Device bytes of one context's request buffers: two FP32 RGB frames, the flow and the occlusion map."""
    return width * height * (2 * 12 + 8 + 1)


def slot_bytes(params: gpm.Params, max_width: int, max_height: int) -> int:
    """gpm_required_bytes of a one-pair context for frames up to max_width x max_height."""
    lib = gpm.load()
    lim = gpm.Limits(max_width, max_height, 1, 0, 0)
    return int(lib.gpm_required_bytes(C.byref(params), C.byref(lim)))


class Admission:
    """HBM-budget bookkeeping of size-class contexts (host logic only; no device calls of its own).

    ``create(cls, budget_left)`` makes a context for size class cls = (width, height) within budget_left bytes
    and returns it, or returns None when the library refuses it with GPM_EBUSY; ``destroy(ctx)`` frees one;
    ``cost(cls)`` is the bytes a context of the class holds."""

    def __init__(self, budget_bytes: int, cost, create, destroy, size_quantum: int = 64, max_active: int = 16):
        self.budget = int(budget_bytes)
        self.cost, self.create, self.destroy = cost, create, destroy
        self.q = int(size_quantum)
        self.max_active = int(max_active)
        self.used = 0                    # bytes held by live contexts, busy and idle
        self.idle: dict = {}             # class -> [context, ...] (most recently used last)
        self.lru: list = []              # idle (class, context) pairs, least recently used first
        self.active = 0
        self.created = self.evicted = self.refused = 0

    def size_class(self, width: int, height: int) -> tuple[int, int]:
        q = self.q
        return (-(-width // q) * q, -(-height // q) * q)

    def acquire(self, width: int, height: int):
        """A context for a width x height pair, or None (GPM_EBUSY: the request waits)."""
        if self.active >= self.max_active:
            return None
        cls = self.size_class(width, height)
        if self.idle.get(cls):
            ctx = self.idle[cls].pop()
            self.lru.remove((cls, ctx))
            self.active += 1
            return ctx
        need = self.cost(cls)
        if need > self.budget:
            raise ValueError(f"a {width}x{height} pair needs {need} bytes, above the whole budget {self.budget}")
        while self.used + need > self.budget and self.lru:
            ocls, octx = self.lru.pop(0)
            self.idle[ocls].remove(octx)
            self.destroy(octx)
            self.used -= self.cost(ocls)
            self.evicted += 1
        if self.used + need > self.budget:
            self.refused += 1
            return None
        ctx = self.create(cls, self.budget - self.used)
        if ctx is None:
            self.refused += 1
            return None
        self.used += need
        self.created += 1
        self.active += 1
        return ctx

    def release(self, cls, ctx, keep: bool = True):
        """A finished request's context: kept idle for its class, or destroyed (keep=False)."""
        self.active -= 1
        if keep:
            self.idle.setdefault(cls, []).append(ctx)
            self.lru.append((cls, ctx))
        else:
            self.destroy(ctx)
            self.used -= self.cost(cls)

    def drain(self):
        """Destroys every idle context."""
        for cls, ctx in self.lru:
            self.destroy(ctx)
            self.used -= self.cost(cls)
        self.idle, self.lru = {}, []


@dataclass
class _Slot:
    cls: tuple
    ctx: gpm.Context
    stream: object
    f1: object
    f2: object
    flow: object
    occ: object
    h_flow: object
    h_occ: object
    h_in: object                   # pinned staging of the request's two frames
    req: Request | None = None
    done: object = None


class Server:
    """Continuous batching of requests under an HBM budget (bytes of context state and request buffers)."""

    def __init__(self, params: gpm.Params, hbm_budget_bytes: int, max_active: int = 16, size_quantum: int = 64):
        import torch
        self.torch = torch
        self.params = params
        self.adm = Admission(hbm_budget_bytes, self._cost, self._create, self._destroy, size_quantum, max_active)
        self.running: list[_Slot] = []
        self.waiting: list[Request] = []
        self._cost_cache: dict = {}
        self._cancel: set = set()

    # ---------------------------------------------------------------- contexts
    def _cost(self, cls) -> int:
        if cls not in self._cost_cache:
            self._cost_cache[cls] = slot_bytes(self.params, *cls) + io_bytes(*cls)
        return self._cost_cache[cls]

    def _create(self, cls, budget_left: int):
        torch = self.torch
        W, H = cls
        st = torch.cuda.Stream()
        try:
            with torch.cuda.stream(st):
                ctx = gpm.Context(self.params, W, H, 1, hbm_budget_bytes=max(1, budget_left - io_bytes(W, H)),
                                  stream=st)
        except gpm.GpmError as e:
            if e.status == gpm.GPM_EBUSY:
                return None
            raise
        with torch.cuda.stream(st):
            f1 = torch.empty(W * H * 3, dtype=torch.float32, device="cuda")
            f2 = torch.empty_like(f1)
            flow = torch.empty(W * H * 2, dtype=torch.float32, device="cuda")
            occ = torch.empty(W * H, dtype=torch.uint8, device="cuda")
        h_flow = torch.empty(W * H * 2, dtype=torch.float32).pin_memory()
        h_occ = torch.empty(W * H, dtype=torch.uint8).pin_memory()
        h_in = torch.empty(2 * W * H * 3, dtype=torch.float32).pin_memory()
        return _Slot(cls, ctx, st, f1, f2, flow, occ, h_flow, h_occ, h_in)

    def _destroy(self, s: _Slot):
        s.stream.synchronize()
        s.ctx.close()

    def close(self):
        for s in self.running:
            s.stream.synchronize()
            self._destroy(s)
        self.running = []
        self.adm.drain()

    @property
    def used_bytes(self) -> int:
        return self.adm.used

    def cancel(self, rid: int):
        """Cancels request rid: it leaves the queue, or its running result is dropped and its context freed."""
        self._cancel.add(rid)

    # ---------------------------------------------------------------- requests
    def _launch(self, s: _Slot, r: Request, t0: float):
        torch = self.torch
        H, W, _ = r.frame1.shape
        n = W * H
        r.t_start = time.perf_counter() - t0
        # host frames -> pinned staging (host copy) -> device, asynchronously on the context's stream
        stage = s.h_in.numpy()
        np.copyto(stage[: 3 * n], r.frame1.reshape(-1))
        np.copyto(stage[3 * n: 6 * n], r.frame2.reshape(-1))
        with torch.cuda.stream(s.stream):
            s.f1[: 3 * n].copy_(s.h_in[: 3 * n], non_blocking=True)
            s.f2[: 3 * n].copy_(s.h_in[3 * n: 6 * n], non_blocking=True)
            f1 = s.f1[: 3 * n].view(H, W, 3)
            f2 = s.f2[: 3 * n].view(H, W, 3)
            s.ctx.match([(f1, f2)], 0, pair_ids=[r.pair_id])
            for level in range(1, self.params.num_scales + 1):
                s.ctx.fit_planes(level)
                s.ctx.match(None, level)
            s.ctx.flow_and_occlusion([s.flow[: 2 * n].view(H, W, 2)], [s.occ[:n].view(H, W)])
            s.h_flow[: 2 * n].copy_(s.flow[: 2 * n], non_blocking=True)
            s.h_occ[:n].copy_(s.occ[:n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s.stream)
        s.req, s.done = r, ev

    def _finish(self, s: _Slot, t0: float):
        r = s.req
        H, W, _ = r.frame1.shape
        n = W * H
        r.t_done = time.perf_counter() - t0
        if r.rid in self._cancel:  # cancelled while it ran: no result, and its context is freed
            r.cancelled = True
            self.adm.release(s.cls, s, keep=False)
        else:
            r.flow = s.h_flow[: 2 * n].numpy().reshape(H, W, 2).copy()
            r.occ = s.h_occ[:n].numpy().reshape(H, W).copy()
            self.adm.release(s.cls, s, keep=True)
        s.req, s.done = None, None

    def poll(self, t0: float) -> int:
        """Finishes completed requests, drops cancelled waiting ones and admits waiting requests in arrival order
        while the budget allows; returns the number running."""
        for s in list(self.running):
            if s.done.query():
                self._finish(s, t0)
                self.running.remove(s)
        kept = []
        for r in self.waiting:
            if r.rid in self._cancel:
                r.cancelled = True
            else:
                kept.append(r)
        self.waiting = kept
        while self.waiting:
            r = self.waiting[0]
            s = self.adm.acquire(*r.size)
            if s is None:
                r.refusals += 1
                break
            self.waiting.pop(0)
            self._launch(s, r, t0)
            self.running.append(s)
        return len(self.running)

    def run(self, requests: list[Request], realtime: bool = True, poll_s: float = 2e-4,
            cancel_at: dict | None = None) -> dict:
        """Serves `requests` (arrival times in seconds); returns latency and throughput statistics.
        cancel_at: {rid: seconds} cancels a request at that time after the start (checked after each pass's
        admissions, so a request cancelled at its own arrival time has started if it was admitted at once)."""
        queue = sorted(requests, key=lambda r: (r.arrival, r.rid))
        cancel_at = dict(cancel_at or {})
        t0 = time.perf_counter()
        i = 0
        peak_used = 0
        while i < len(queue) or self.waiting or self.running:
            now = time.perf_counter() - t0
            while i < len(queue) and (queue[i].arrival <= now or not realtime):
                self.waiting.append(queue[i])
                i += 1
            n = self.poll(t0)
            for rid, tc in list(cancel_at.items()):  # after the admissions of this pass
                if tc <= now:
                    self.cancel(rid)
                    del cancel_at[rid]
            peak_used = max(peak_used, self.adm.used)
            if n and (self.waiting or i == len(queue)):
                time.sleep(poll_s)
            elif not self.waiting and i < len(queue):
                time.sleep(max(0.0, min(queue[i].arrival - (time.perf_counter() - t0), 1e-3)))
        done = [r for r in requests if not r.cancelled]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        first = min(r.arrival for r in requests)
        last = max(r.t_done for r in done) if done else first
        return {"requests": len(done), "cancelled": len(requests) - len(done),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "pairs_per_s": len(done) / max(last - first, 1e-9),
                "wall_s": last, "peak_used_bytes": peak_used, "budget_bytes": self.adm.budget,
                "contexts_created": self.adm.created, "contexts_evicted": self.adm.evicted,
                "admissions_refused": self.adm.refused}


def poisson_trace(rate_hz: float, duration_s: float, pool: list, seed: int = 0, max_requests: int | None = None
                  ) -> list[Request]:
    """Seeded Poisson arrivals; each request takes a pair from `pool` (list of (frame1, frame2))."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while max_requests is None or len(out) < max_requests:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        f1, f2 = pool[int(rng.integers(len(pool)))]
        out.append(Request(rid=len(out), arrival=t, frame1=f1, frame2=f2, pair_id=len(out)))
    return out


def serving_specs(n: int, seed: int = 0) -> list[dict]:
    """Scene recipes of the serving workload: log-uniform sizes 320x240 to 1920x1080, 4-7 layers, motion up to
    width / 13 px (25 px at 320, 128 px at 1664 and above), so that the occluded fraction stays near the
    benchmark scenes' (about 10 %, 4-14 % over the 32-scene pool of seed 0).  Each is a keyword dict for
    scene.make_scene."""
    rng = np.random.default_rng(seed + 7)
    out = []
    for k, (w, h) in enumerate(log_uniform_sizes(n, seed=seed)):
        out.append(dict(width=w, height=h, seed=3000 + seed * 100 + k, n_layers=int(rng.integers(4, 8)),
                        max_disp=float(min(128.0, w / 13.0)), affine=False, area_frac=(0.02, 0.08)))
    return out


def log_uniform_sizes(n: int, lo=(320, 240), hi=(1920, 1080), seed: int = 0) -> list[tuple[int, int]]:
    """Frame sizes whose pixel count is log-uniform between lo and hi (16:9 to 4:3 aspect between the ends)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a = rng.uniform(0, 1)
        w = int(round(math.exp(math.log(lo[0]) + a * (math.log(hi[0]) - math.log(lo[0])))))
        h = int(round(math.exp(math.log(lo[1]) + a * (math.log(hi[1]) - math.log(lo[1])))))
        out.append((w, h))
    return out
