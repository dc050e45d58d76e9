"""Serving: Poisson traces and frame sizes (CPU), and on the GPU the
continuous-batching loop -- each result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_1804_03787_gb300 import scene, serve


def test_poisson_trace_is_seeded_and_has_the_rate():
    pool = [(np.zeros((4, 4, 3), np.float32), np.zeros((4, 4, 3), np.float32))]
    a = serve.poisson_trace(200.0, 5.0, pool, seed=3)
    b = serve.poisson_trace(200.0, 5.0, pool, seed=3)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert 850 < len(a) < 1150
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0


def test_log_uniform_sizes_span_the_range():
    sizes = serve.log_uniform_sizes(2000, seed=1)
    w = np.array([s[0] for s in sizes])
    h = np.array([s[1] for s in sizes])
    assert w.min() >= 320 and w.max() <= 1920 and h.min() >= 240 and h.max() <= 1080
    # log-uniform pixel count: the median sits near the geometric mean
    px = w * h
    gm = np.sqrt(320 * 240 * 1920 * 1080)
    assert 0.7 * gm < np.median(px) < 1.4 * gm


class _FakeLib:
    """Stands in for context creation: records creations and destructions; refuses (GPM_EBUSY) on request."""

    def __init__(self, refuse=False):
        self.made, self.gone, self.refuse = [], [], refuse

    def cost(self, cls):
        return cls[0] * cls[1]

    def create(self, cls, left):
        if self.refuse or self.cost(cls) > left:
            return None
        c = ("ctx", cls, len(self.made))
        self.made.append(c)
        return c

    def destroy(self, c):
        self.gone.append(c)


def _adm(budget, refuse=False, active=16):
    f = _FakeLib(refuse)
    return serve.Admission(budget, f.cost, f.create, f.destroy, size_quantum=64, max_active=active), f


def test_admission_rounds_sizes_to_classes():
    a, _ = _adm(10**9)
    assert a.size_class(320, 240) == (320, 256)
    assert a.size_class(321, 1) == (384, 64)
    assert a.size_class(1920, 1080) == (1920, 1088)


def test_admission_by_each_request_size_within_the_budget():
    """Small requests are admitted by their own size: four 64x64 contexts fit where one 128x128 would."""
    a, f = _adm(4 * 64 * 64)
    got = [a.acquire(60, 60) for _ in range(4)]
    assert all(g is not None for g in got) and a.used == 4 * 64 * 64
    assert a.acquire(10, 10) is None and a.refused == 1      # full: GPM_EBUSY, the request waits
    a.release((64, 64), got[0])
    assert a.acquire(64, 64) is got[0] and len(f.made) == 4  # the idle context of its class is reused


def test_admission_evicts_idle_contexts_least_recently_used_first():
    a, f = _adm(4 * 64 * 64)
    x = a.acquire(64, 64)     # 1 unit
    y = a.acquire(128, 64)    # 2 units
    a.release((128, 64), y)
    a.release((64, 64), x)    # x used last
    w = a.acquire(64, 128)    # 2 units: only y (least recently used) has to go
    assert w is not None and f.gone == [y] and a.evicted == 1 and a.used == 3 * 64 * 64
    a.release((64, 128), w)
    z = a.acquire(128, 128)   # 4 units: every idle context goes, x first
    assert z is not None and f.gone == [y, x, w] and a.evicted == 3 and a.used == 128 * 128


def test_admission_waits_while_busy_contexts_hold_the_budget():
    a, f = _adm(2 * 64 * 64)
    x = a.acquire(64, 64)
    assert a.acquire(128, 64) is None  # x is busy: nothing to evict
    a.release((64, 64), x, keep=False)  # a cancelled request: its context is freed
    assert f.gone == [x] and a.used == 0
    assert a.acquire(128, 64) is not None


def test_admission_refused_by_the_library_is_ebusy():
    a, f = _adm(10**9, refuse=True)
    assert a.acquire(64, 64) is None and a.refused == 1 and a.used == 0 and a.active == 0


def test_admission_caps_concurrent_requests_and_rejects_oversize():
    a, _ = _adm(10**9, active=2)
    assert a.acquire(64, 64) is not None and a.acquire(64, 64) is not None
    assert a.acquire(64, 64) is None
    b, _ = _adm(100)
    with pytest.raises(ValueError):
        b.acquire(64, 64)


def test_admission_drain_frees_everything_idle():
    a, f = _adm(10**9)
    xs = [a.acquire(64 * k, 64) for k in (1, 2, 3)]
    for k, x in zip((1, 2, 3), xs):
        a.release((64 * k, 64), x)
    a.drain()
    assert sorted(f.gone) == sorted(xs) and a.used == 0


def _pool():
    sizes = [(96, 72), (128, 96), (80, 64), (112, 80), (64, 48)]
    pool = []
    for k, (w, h) in enumerate(sizes):
        s = scene.make_scene(w, h, seed=40 + k, n_layers=2, max_disp=5.0)
        pool.append((s.frame1, s.frame2))
    return pool


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    import torch
    from paper_1804_03787_gb300 import gpm
    assert torch.cuda.is_available()
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=64)
    pool = _pool()
    srv = serve.Server(gp, hbm_budget_bytes=3 * serve.slot_bytes(gp, 128, 128) + (64 << 20), max_active=4)
    alone = []
    for k, (f1, f2) in enumerate(pool):
        r = serve.Request(rid=k, arrival=0.0, frame1=f1, frame2=f2, pair_id=100 + k)
        srv.run([r], realtime=False)
        alone.append((r.flow, r.occ))
    mix = [serve.Request(rid=k, arrival=0.001 * k, frame1=f1, frame2=f2, pair_id=100 + k)
           for k, (f1, f2) in enumerate(pool)]
    stats = srv.run(mix, realtime=False)
    for k, r in enumerate(mix):
        np.testing.assert_array_equal(r.flow, alone[k][0])
        np.testing.assert_array_equal(r.occ, alone[k][1])
    assert stats["requests"] == 5 and stats["p50_ms"] <= stats["p99_ms"] and stats["pairs_per_s"] > 0
    assert stats["peak_used_bytes"] <= stats["budget_bytes"]
    srv.close()
    assert srv.used_bytes == 0


@pytest.mark.gpu
def test_cancelled_request_frees_its_context():
    """A budget that holds one context: the running request is cancelled, its context is freed when its kernels
    finish (no result), and the next request -- which could not be admitted meanwhile -- then runs; a cancelled
    queued request never runs."""
    import torch
    from paper_1804_03787_gb300 import gpm
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=64)
    pool = _pool()
    one = serve.slot_bytes(gp, 128, 128) + serve.io_bytes(128, 128)
    srv = serve.Server(gp, hbm_budget_bytes=one + one // 2, max_active=4)
    reqs = [serve.Request(rid=k, arrival=0.0, frame1=pool[1][0], frame2=pool[1][1], pair_id=k) for k in range(3)]
    stats = srv.run(reqs, realtime=True, cancel_at={0: 0.0, 2: 0.0})
    assert reqs[0].cancelled and reqs[0].flow is None and reqs[0].t_start >= 0  # it had started
    assert reqs[2].cancelled and reqs[2].t_start < 0                             # it never started
    assert not reqs[1].cancelled and reqs[1].flow is not None
    assert reqs[1].refusals >= 1 and stats["cancelled"] == 2 and stats["requests"] == 1
    assert stats["peak_used_bytes"] <= one + one // 2
    srv.close()
    assert srv.used_bytes == 0
