"""Batched form: many frame pairs of mixed sizes per step.

The pairs go to one or more gpm contexts, one CUDA stream each, balanced by
pixel count.  Inside a context the pair index is on the device: every stage
is one launch per eight of the context's pairs (blockIdx.z = pair), so a
context of eight pairs makes the same ~190 launches as one of a single pair.  Each stream's whole pipeline (every scale, both directions,
flow and occlusion) is captured once into a CUDA graph and replayed as a
single launch per step.  The number of streams and the PatchMatch launch
shape (blocks per SM) are picked by a small autotuner that times replays of
each candidate, its choice cached by the batch's frame sizes, patch radius
and storage type.

Every pair's result depends only on its frames, its pair id and the
parameters, so the grouping changes nothing but the speed.
"""
from __future__ import annotations

import numpy as np

from . import gpm

# Batched workload: sizes drawn uniformly from these (width, height) pairs.
BATCH_SIZES = ((256, 192), (512, 384), (1024, 436), (1280, 720))


class BatchRunner:
    """Runs the whole method for a fixed set of device-resident frame pairs."""

    def __init__(self, params: gpm.Params, frames, pair_ids, streams: int = 4, graph: bool = True):
        import torch
        self.torch = torch
        self.params = params
        n = len(frames)
        self.n = n
        self.pair_ids = list(pair_ids)
        px = [f1.shape[0] * f1.shape[1] for f1, _ in frames]
        groups = [[] for _ in range(max(1, min(streams, n)))]
        load = [0] * len(groups)
        for i in sorted(range(n), key=lambda i: (-px[i], i)):  # largest first onto the least loaded stream
            g = int(np.argmin(load))
            groups[g].append(i)
            load[g] += px[i]
        self.groups = []
        for idx in groups:
            idx = sorted(idx)
            st = torch.cuda.Stream()
            mw = max(frames[i][0].shape[1] for i in idx)
            mh = max(frames[i][0].shape[0] for i in idx)
            with torch.cuda.stream(st):
                ctx = gpm.Context(params, mw, mh, max_pairs=len(idx), stream=st)
                dev = [(torch.from_numpy(np.ascontiguousarray(frames[i][0])).cuda(),
                        torch.from_numpy(np.ascontiguousarray(frames[i][1])).cuda()) for i in idx]
                flows = [torch.empty((f1.shape[0], f1.shape[1], 2), dtype=torch.float32, device="cuda")
                         for f1, _ in dev]
                occs = [torch.empty((f1.shape[0], f1.shape[1]), dtype=torch.uint8, device="cuda") for f1, _ in dev]
            self.groups.append({"stream": st, "ctx": ctx, "idx": idx, "dev": dev, "flows": flows, "occs": occs,
                                "graph": None})
        torch.cuda.synchronize()
        if graph:
            self.capture()

    def _enqueue(self, G):
        ctx = G["ctx"]
        ctx.match(G["dev"], 0, pair_ids=[self.pair_ids[i] for i in G["idx"]])
        for level in range(1, self.params.num_scales + 1):
            ctx.fit_planes(level)
            ctx.match(None, level)
        ctx.flow_and_occlusion(G["flows"], G["occs"])

    def capture(self):
        """One eager run per stream (sizes, kernel attributes), then a CUDA graph of the pipeline."""
        torch = self.torch
        for G in self.groups:
            with torch.cuda.stream(G["stream"]):
                self._enqueue(G)
            G["stream"].synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=G["stream"]):
                self._enqueue(G)
            G["graph"] = g
        torch.cuda.synchronize()

    def run(self):
        """Enqueues one pass over all pairs; the current stream waits for every group."""
        torch = self.torch
        cur = torch.cuda.current_stream()
        for G in self.groups:
            G["stream"].wait_stream(cur)
            with torch.cuda.stream(G["stream"]):
                if G["graph"] is not None:
                    G["graph"].replay()
                else:
                    self._enqueue(G)
        for G in self.groups:
            cur.wait_stream(G["stream"])

    def time(self, reps: int = 1) -> float:
        """Seconds per pass (CUDA events on the current stream around `reps` passes)."""
        torch = self.torch
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            self.run()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3 / reps

    def results(self):
        """(flow, occlusion) per pair, as host arrays in the input order."""
        out = [None] * self.n
        for G in self.groups:
            for j, i in enumerate(G["idx"]):
                out[i] = (G["flows"][j].cpu().numpy(), G["occs"][j].cpu().numpy())
        return out

    def close(self):
        for G in self.groups:
            G["graph"] = None
            G["ctx"].close()
        self.groups = []


# Autotuner choices, keyed by (frame sizes, patch radius, storage type).
_TUNE_CACHE: dict = {}


def with_launch_shape(params: gpm.Params, blocks_per_sm: int) -> gpm.Params:
    """A copy of params with the PatchMatch launch shape set (results do not depend on it)."""
    p = type(params).from_buffer_copy(params)
    p.sweep_blocks_per_sm = blocks_per_sm
    return p


def autotune(params: gpm.Params, frames, pair_ids, streams=(1, 2, 4), blocks_per_sm=(4, 8), reps: int = 1,
             cache: dict | None = None):
    """Times a captured runner for each (stream count, PatchMatch blocks per SM); returns the fastest pair and
    {candidate: seconds per pass}.  The choice is cached by the batch's frame sizes, patch radius and storage."""
    import torch
    cache = _TUNE_CACHE if cache is None else cache
    key = (tuple(sorted((int(f1.shape[1]), int(f1.shape[0])) for f1, _ in frames)), int(params.patch_radius),
           int(params.storage))
    if key in cache:
        return cache[key]
    times = {}
    for s in streams:
        for b in blocks_per_sm:
            r = BatchRunner(with_launch_shape(params, b), frames, pair_ids, streams=s, graph=True)
            r.run()
            times[(s, b)] = r.time(reps)
            r.close()
            del r
            torch.cuda.empty_cache()
    best = min(times, key=lambda k: (times[k], k))
    cache[key] = (best, times)
    return best, times


def epe(flow: np.ndarray, gt: np.ndarray, mask: np.ndarray | None = None) -> float:
    """Mean end-point error over the pixels where `mask` is true (all pixels if None)."""
    e = np.sqrt(((flow - gt) ** 2).sum(-1))
    return float(e.mean() if mask is None else e[mask].mean())


def batch_specs(distinct: int = 16, seed: int = 0, sizes=BATCH_SIZES):
    """Scene recipes of the batched workload: sizes uniform over `sizes`, 3-8 layers, motion up to 96 px.
    Each is a keyword dict for scene.make_scene."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(distinct):
        w, h = sizes[int(rng.integers(len(sizes)))]
        out.append(dict(width=w, height=h, seed=1000 + seed * 100 + k, n_layers=int(rng.integers(3, 9)),
                        max_disp=96.0, affine=False, area_frac=(0.02, 0.08)))
    return out


def make_scene_from_spec(spec):
    from . import scene
    return scene.make_scene(**spec)


def make_scenes(specs, workers: int = 0):
    """Renders the scenes, in parallel processes (spawned, so safe after CUDA is initialised) if workers > 1."""
    if workers <= 1 or len(specs) <= 1:
        return [make_scene_from_spec(s) for s in specs]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=min(workers, len(specs)), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(make_scene_from_spec, specs))
