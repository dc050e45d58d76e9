"""Python binding of the C ABI in ``include/gpm.h`` (ctypes, argument
marshalling only).

Every step of the method runs inside ``libgpm.so``; PyTorch only provides
device memory (the context's buffers come from its caching allocator through
the ABI's allocator callbacks) and the CUDA stream.  There is no CPU fallback:
loading fails loudly when the library or a GPU is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

MAX_SCALES = 8
MI = 12
GPM_OK, GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA, GPM_EBUSY, GPM_EINTERNAL = 0, 1, 2, 3, 5, 6
GPM_F32, GPM_F16, GPM_BF16 = 0, 1, 2
(NNF, COST, MODELS, MODEL_INFO, LABELS, LEVEL_LABELS, STAGE1_LABELS, CUES, FRAMES, TENT_LABELS) = range(10)

# every symbol the header declares (checked by the CPU test suite)
EXPORTED = ["gpm_default_params", "gpm_create", "gpm_destroy", "gpm_required_bytes", "gpm_match",
            "gpm_fit_planes", "gpm_flow_and_occlusion", "gpm_sync", "gpm_state_bytes", "gpm_export",
            "gpm_import", "gpm_status_string", "gpm_last_error", "gpm_launch_count", "gpm_profile_enable",
            "gpm_profile_select", "gpm_profile_read", "gpm_ingest_noalloc", "gpm_fp32_peak_probe"]
(COUNT_SWEEP0, COUNT_SWEEP_PLANE, COUNT_RANSAC, COUNT_INIT, COUNT_SWEEP0_TAPS, COUNT_SWEEP_PLANE_TAPS,
 COUNT_SWEEP0_PRUNED, COUNT_RANSAC_FP64, COUNT_RANSAC_LOOSE) = range(9)
COUNTERS = 9
PROF_CLASSES = ["ingest", "pm_init", "pm_sweep", "pm_sweep_plane", "pm_recost", "ransac", "assign", "cues",
                "many_to_one", "merge", "lists", "fill", "final"]


class GpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Params(C.Structure):
    _fields_ = [("patch_radius", C.c_int32), ("num_scales", C.c_int32), ("cell_size", C.c_int32 * MAX_SCALES),
                ("pm_iters", C.c_int32), ("num_hyp", C.c_int32), ("min_inliers", C.c_int32),
                ("fill_iters", C.c_int32), ("gain_normalize", C.c_int32), ("pm_init", C.c_int32),
                ("storage", C.c_int32), ("equalize", C.c_int32), ("eps", C.c_float), ("ransac_px", C.c_float),
                ("fb_px", C.c_float), ("eta", C.c_float), ("kappa", C.c_float), ("beta", C.c_float),
                ("occ_thresh", C.c_float), ("scale_min", C.c_float), ("scale_max", C.c_float),
                ("census", C.c_int32), ("seed", C.c_uint64), ("interp", C.c_int32),
                ("sweep_blocks_per_sm", C.c_int32)]


class Limits(C.Structure):
    _fields_ = [("max_width", C.c_int32), ("max_height", C.c_int32), ("max_pairs", C.c_int32),
                ("reserved", C.c_int32), ("hbm_budget_bytes", C.c_size_t)]


class Pair(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("row_stride", C.c_int64),
                ("frame1", C.c_void_p), ("frame2", C.c_void_p), ("pair_id", C.c_uint32), ("dtype", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_lib = None


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libgpm.so")


def load(build: bool = True) -> C.CDLL:
    """Loads libgpm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        from . import build_lib
        build_lib.build()
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1804_03787_gb300.build_lib.build()")
    L = C.CDLL(path)
    P = C.POINTER
    sig = {
        "gpm_default_params": (None, [P(Params)]),
        "gpm_create": (C.c_int, [P(Params), P(Limits), ALLOC_FN, FREE_FN, C.c_void_p, C.c_void_p, P(C.c_void_p)]),
        "gpm_destroy": (C.c_int, [C.c_void_p]),
        "gpm_required_bytes": (C.c_size_t, [P(Params), P(Limits)]),
        "gpm_match": (C.c_int, [C.c_void_p, P(Pair), C.c_int32, C.c_int32]),
        "gpm_fit_planes": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
        "gpm_flow_and_occlusion": (C.c_int, [C.c_void_p, C.c_int32, P(C.c_void_p), P(C.c_void_p)]),
        "gpm_sync": (C.c_int, [C.c_void_p]),
        "gpm_state_bytes": (C.c_size_t, [C.c_void_p, C.c_int32, C.c_int32]),
        "gpm_export": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
        "gpm_import": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32]),
        "gpm_status_string": (C.c_char_p, [C.c_int]),
        "gpm_last_error": (C.c_char_p, [C.c_void_p]),
        "gpm_launch_count": (C.c_uint64, [C.c_void_p]),
        "gpm_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
        "gpm_profile_select": (C.c_int, [C.c_void_p, C.c_uint32, C.c_int32]),
        "gpm_profile_read": (C.c_int, [C.c_void_p, P(C.c_double), P(C.c_uint64), P(C.c_uint64)]),
        "gpm_ingest_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_int32,
                                         C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
        "gpm_fp32_peak_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def fp32_peak_probe(blocks: int, iters: int, sink, stream=None) -> int:
    """Launches the FP32 FMA probe (gpm_fp32_peak_probe) on the stream; returns the lane operations it executes.
    sink: a CUDA float32 tensor of at least blocks x 256 elements."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    r = load().gpm_fp32_peak_probe(blocks, iters, C.c_void_p(sink.data_ptr()), C.c_void_p(st.cuda_stream))
    if r != GPM_OK:
        raise GpmError(r, "gpm_fp32_peak_probe failed")
    return blocks * 256 * iters * 512


def default_params(**kw) -> Params:
    p = Params()
    load().gpm_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "cells":
            p.num_scales = len(v)
            for i, s in enumerate(v):
                p.cell_size[i] = s
        else:
            setattr(p, k, v)
    return p


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libgpm needs a CUDA device; none is visible")
    return torch


class Context:
    """A gpm context: device state for up to ``max_pairs`` frame pairs."""

    def __init__(self, params: Params, max_width: int, max_height: int, max_pairs: int = 1,
                 hbm_budget_bytes: int = 0, stream=None):
        torch = _torch()
        self._torch = torch
        self.lib = load()
        self.params = params
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._blocks = {}

        def _alloc(user, nbytes, stream):
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            self._blocks[t.data_ptr()] = t
            return t.data_ptr()

        def _free(user, ptr, stream):
            self._blocks.pop(ptr, None)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        lim = Limits(max_width, max_height, max_pairs, 0, hbm_budget_bytes)
        self.limits = lim
        h = C.c_void_p()
        st = self.lib.gpm_create(C.byref(params), C.byref(lim), self._alloc_cb, self._free_cb, None,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != GPM_OK:
            raise GpmError(st, f"gpm_create failed: {self.lib.gpm_status_string(st).decode()}")
        self.h = h
        self._pairs = None
        self._n = 0

    # ------------------------------------------------------------ stages
    def _check(self, st: int, what: str):
        if st != GPM_OK:
            msg = self.lib.gpm_last_error(self.h).decode()
            raise GpmError(st, f"{what}: {self.lib.gpm_status_string(st).decode()}: {msg}")

    def match(self, frames, level: int = 0, pair_ids=None):
        """frames: list of (frame1, frame2) CUDA HxWx3 tensors, float32, float16 or bfloat16 (both frames of a pair
        alike; level 0 only)."""
        if level == 0:
            torch = self._torch
            kinds = {torch.float32: GPM_F32, torch.float16: GPM_F16, torch.bfloat16: GPM_BF16}
            n = len(frames)
            arr = (Pair * n)()
            self._keep = []
            for i, (f1, f2) in enumerate(frames):
                f1 = f1.contiguous()
                f2 = f2.contiguous()
                if f1.dtype != f2.dtype or f1.dtype not in kinds:
                    raise ValueError("frames must both be float32, float16 or bfloat16")
                self._keep += [f1, f2]
                H, W, _ = f1.shape
                arr[i] = Pair(W, H, 3 * W, f1.data_ptr(), f2.data_ptr(),
                              (pair_ids[i] if pair_ids is not None else i) & 0xFFFFFFFF, kinds[f1.dtype])
                self._pairs = [(W, H) for (W, H) in [(f.shape[1], f.shape[0]) for f, _ in frames]]
            self._check(self.lib.gpm_match(self.h, arr, n, 0), "gpm_match")
            self._n = n
        else:
            self._check(self.lib.gpm_match(self.h, None, self._n, level), "gpm_match")

    def fit_planes(self, level: int):
        self._check(self.lib.gpm_fit_planes(self.h, self._n, level), "gpm_fit_planes")

    def flow_and_occlusion(self, flows=None, occs=None):
        torch = self._torch
        if flows is None:
            flows = [torch.empty((H, W, 2), dtype=torch.float32, device="cuda") for (W, H) in self._pairs]
            occs = [torch.empty((H, W), dtype=torch.uint8, device="cuda") for (W, H) in self._pairs]
        fp = (C.c_void_p * self._n)(*[f.data_ptr() for f in flows])
        op = (C.c_void_p * self._n)(*[o.data_ptr() for o in occs])
        self._check(self.lib.gpm_flow_and_occlusion(self.h, self._n, fp, op), "gpm_flow_and_occlusion")
        return flows, occs

    def run(self, frames, pair_ids=None):
        """Whole method for a list of frame pairs: returns (flows, occlusions)."""
        self.match(frames, 0, pair_ids)
        for l in range(1, self.params.num_scales + 1):
            self.fit_planes(l)
            self.match(None, l)
        return self.flow_and_occlusion()

    def sync(self):
        self._check(self.lib.gpm_sync(self.h), "gpm_sync")

    def launch_count(self) -> int:
        return int(self.lib.gpm_launch_count(self.h))

    def profile_enable(self, on: bool = True):
        self._check(self.lib.gpm_profile_enable(self.h, 1 if on else 0), "gpm_profile_enable")

    def profile_select(self, classes, count_evals: bool = False):
        """Brackets only the launches of the named kernel classes (names of PROF_CLASSES) with events."""
        mask = 0
        for name in classes:
            mask |= 1 << PROF_CLASSES.index(name)
        self._check(self.lib.gpm_profile_select(self.h, mask, 1 if count_evals else 0), "gpm_profile_select")

    def profile_read(self):
        """{class: (ms, launches)} and the work counts (a tuple indexed by the COUNT_* constants: level-0 sweep
        evaluations, plane-level sweep evaluations, RANSAC residual tests, init / recost evaluations, taps summed by
        the level-0 sweeps, taps summed by the plane-level sweeps, level-0 candidates rejected by the patch-sum bound,
        RANSAC tests decided in FP64, RANSAC hypotheses tested with per-match bounds); clears them."""
        k = len(PROF_CLASSES)
        ms = (C.c_double * k)()
        ln = (C.c_uint64 * k)()
        ev = (C.c_uint64 * COUNTERS)()
        self._check(self.lib.gpm_profile_read(self.h, ms, ln, ev), "gpm_profile_read")
        return {PROF_CLASSES[i]: (ms[i], int(ln[i])) for i in range(k)}, tuple(int(e) for e in ev)

    # ------------------------------------------------------------ state
    def export(self, what: int, pair: int = 0):
        """Exports state as CPU numpy arrays (synchronises)."""
        torch = self._torch
        nb = self.lib.gpm_state_bytes(self.h, pair, what)
        if nb == 0:
            raise GpmError(GPM_EINVAL, "nothing to export")
        buf = torch.empty(int(nb), dtype=torch.uint8, device="cuda")
        self._check(self.lib.gpm_export(self.h, pair, what, C.c_void_p(buf.data_ptr())), "gpm_export")
        self.sync()
        raw = buf.cpu().numpy()
        W, H = self._pairs[pair]
        n = W * H
        if what == NNF:
            return raw.view(np.int32).reshape(2, n, 2)
        if what == COST:
            return raw.view(np.float32).reshape(2, n)
        if what == MODELS:
            return raw.view(np.float64).reshape(2, -1, 9)
        if what == MODEL_INFO:
            return raw.view(np.int32).reshape(2, -1, MI)
        if what in (LABELS, LEVEL_LABELS, STAGE1_LABELS, TENT_LABELS):
            m = raw[: 2 * n * 4].view(np.int32).reshape(2, n)
            L = raw[2 * n * 4: 2 * n * 8].view(np.float32).reshape(2, n)
            a = (2 * n * 8 + 7) // 8 * 8
            f = raw[a: a + 2 * n * 16].view(np.float64).reshape(2, n, 2)
            return m, L, f
        if what == CUES:
            return raw.reshape(2, n)
        if what == FRAMES:
            return raw.view(np.float32).reshape(2, H, W, 4)
        raise ValueError(what)

    def import_state(self, what: int, data, level: int, pair: int = 0, after_fit: bool = False):
        """Imports state that belongs after gpm_match(level), or after gpm_fit_planes(level) with after_fit."""
        torch = self._torch
        if what in (LABELS,):
            m, L, f = data
            n = m.shape[1]
            a = (2 * n * 8 + 7) // 8 * 8
            raw = np.zeros(a + 2 * n * 16, np.uint8)
            raw[: 2 * n * 4] = np.ascontiguousarray(m, np.int32).view(np.uint8).reshape(-1)
            raw[2 * n * 4: 2 * n * 8] = np.ascontiguousarray(L, np.float32).view(np.uint8).reshape(-1)
            raw[a:] = np.ascontiguousarray(f, np.float64).view(np.uint8).reshape(-1)
        else:
            raw = np.ascontiguousarray(data).view(np.uint8).reshape(-1)
        stage = 2 * level - 1 if after_fit else 2 * level
        self.import_state_raw(what, raw, stage, pair, packed=True)
        self.sync()

    def import_state_raw(self, what: int, data, stage: int, pair: int = 0, packed: bool = False):
        """gpm_import at a raw stage number, without the synchronising check (device consistency checks are
        then reported by the next sync)."""
        torch = self._torch
        if what == LABELS and not packed:
            m, L, f = data
            n = m.shape[1]
            a = (2 * n * 8 + 7) // 8 * 8
            raw = np.zeros(a + 2 * n * 16, np.uint8)
            raw[: 2 * n * 4] = np.ascontiguousarray(m, np.int32).view(np.uint8).reshape(-1)
            raw[2 * n * 4: 2 * n * 8] = np.ascontiguousarray(L, np.float32).view(np.uint8).reshape(-1)
            raw[a:] = np.ascontiguousarray(f, np.float64).view(np.uint8).reshape(-1)
        else:
            raw = np.ascontiguousarray(data).view(np.uint8).reshape(-1)
        buf = torch.from_numpy(raw.copy()).to("cuda")
        self._check(self.lib.gpm_import(self.h, pair, what, C.c_void_p(buf.data_ptr()), stage), "gpm_import")
        self._import_keep = buf

    def close(self):
        if getattr(self, "h", None):
            self.lib.gpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
