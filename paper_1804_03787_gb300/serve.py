"""Serving: a continuous-batching request loop over the C ABI.

Frame pairs of different sizes arrive over time.  Each admitted request gets
a slot -- a gpm context with its own CUDA stream and device buffers sized for
the largest frame -- so requests that arrive while others run are admitted as
soon as a slot is free and their kernels overlap on the GPU.  The number of
slots is set by an HBM budget (gpm_required_bytes per slot).  Pyramids of
state (NNF, planes, labels) stay in the slot's device memory for the life of
the request; only the frames go in and the flow and occlusion map come out.

Every request's result depends only on its frames, its pair id and the
parameters: the same alone and in any mix (tests/test_serve.py checks this).
"""
from __future__ import annotations

import ctypes as C
import math
import time
from dataclasses import dataclass, field

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

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


@dataclass
class _Slot:
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


def slot_bytes(params: gpm.Params, max_width: int, max_height: int) -> int:
    lib = gpm.load()
    lim = gpm.Limits(max_width, max_height, 1, 0, 0)
    return int(lib.gpm_required_bytes(C.byref(params), C.byref(lim)))


class Server:
    """Continuous batching over `slots` device slots (at most `hbm_budget_bytes` of state)."""

    def __init__(self, params: gpm.Params, max_width: int, max_height: int, hbm_budget_bytes: int,
                 max_slots: int = 64):
        import torch
        self.torch = torch
        self.params = params
        self.W, self.H = max_width, max_height
        per = slot_bytes(params, max_width, max_height) + max_width * max_height * (2 * 12 + 9)
        n = int(max(1, min(max_slots, hbm_budget_bytes // per)))
        self.slots = []
        for _ in range(n):
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                ctx = gpm.Context(params, max_width, max_height, 1, stream=st)
                f1 = torch.empty(max_width * max_height * 3, dtype=torch.float32, device="cuda")
                f2 = torch.empty_like(f1)
                flow = torch.empty(max_width * max_height * 2, dtype=torch.float32, device="cuda")
                occ = torch.empty(max_width * max_height, dtype=torch.uint8, device="cuda")
            h_flow = torch.empty(max_width * max_height * 2, dtype=torch.float32).pin_memory()
            h_occ = torch.empty(max_width * max_height, dtype=torch.uint8).pin_memory()
            h_in = torch.empty(2 * max_width * max_height * 3, dtype=torch.float32).pin_memory()
            self.slots.append(_Slot(ctx, st, f1, f2, flow, occ, h_flow, h_occ, h_in))
        self.per_slot_bytes = per
        torch.cuda.synchronize()

    def close(self):
        for s in self.slots:
            s.ctx.close()
        self.slots = []

    def _launch(self, s: _Slot, r: Request, t0: float):
        torch = self.torch
        H, W, _ = r.frame1.shape
        n = W * H
        r.t_start = time.perf_counter() - t0
        # host frames -> pinned staging (host copy) -> device, asynchronously on the slot's stream
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
        r.flow = s.h_flow[: 2 * n].numpy().reshape(H, W, 2).copy()
        r.occ = s.h_occ[:n].numpy().reshape(H, W).copy()
        s.req, s.done = None, None

    def run(self, requests: list[Request], realtime: bool = True, poll_s: float = 2e-4) -> dict:
        """Serves `requests` (arrival times in seconds); returns latency and throughput statistics."""
        for r in requests:
            if r.frame1.shape[0] > self.H or r.frame1.shape[1] > self.W:
                raise ValueError(f"request {r.rid} is larger than the slots ({self.W}x{self.H})")
        queue = sorted(requests, key=lambda r: (r.arrival, r.rid))
        waiting: list[Request] = []
        t0 = time.perf_counter()
        i = 0
        busy = 0
        while i < len(queue) or waiting or busy:
            now = time.perf_counter() - t0
            while i < len(queue) and (queue[i].arrival <= now or not realtime):
                waiting.append(queue[i])
                i += 1
            for s in self.slots:
                if s.req is not None and s.done.query():
                    self._finish(s, t0)
                    busy -= 1
            for s in self.slots:
                if not waiting:
                    break
                if s.req is None:
                    self._launch(s, waiting.pop(0), t0)
                    busy += 1
            if busy == len(self.slots) or (not waiting and busy):
                time.sleep(poll_s)
            elif not waiting and i < len(queue):
                time.sleep(max(0.0, min(queue[i].arrival - (time.perf_counter() - t0), 1e-3)))
        lat = np.array([r.latency for r in requests])
        first = min(r.arrival for r in requests)
        last = max(r.t_done for r in requests)
        return {"requests": len(requests), "slots": len(self.slots), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "pairs_per_s": len(requests) / (last - first), "wall_s": last}


def poisson_trace(rate_hz: float, duration_s: float, pool: list, seed: int = 0) -> list[Request]:
    """Seeded Poisson arrivals; each request takes a pair from `pool` (list of (frame1, frame2))."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        f1, f2 = pool[int(rng.integers(len(pool)))]
        out.append(Request(rid=len(out), arrival=t, frame1=f1, frame2=f2, pair_id=len(out)))
    return out


def serving_specs(n: int, seed: int = 0) -> list[dict]:
    """Scene recipes of the serving workload: log-uniform sizes 320x240 to 1920x1080, 4-10 layers, motion up
    to 128 px.  Each is a keyword dict for scene.make_scene."""
    rng = np.random.default_rng(seed + 7)
    out = []
    for k, (w, h) in enumerate(log_uniform_sizes(n, seed=seed)):
        out.append(dict(width=w, height=h, seed=3000 + seed * 100 + k, n_layers=int(rng.integers(4, 11)),
                        max_disp=128.0, affine=False, area_frac=(0.02, 0.08)))
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
