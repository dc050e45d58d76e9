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


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    import torch
    from paper_1804_03787_gb300 import gpm
    assert torch.cuda.is_available()
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=64)
    sizes = [(96, 72), (128, 96), (80, 64), (112, 80), (64, 48)]
    pool = []
    for k, (w, h) in enumerate(sizes):
        s = scene.make_scene(w, h, seed=40 + k, n_layers=2, max_disp=5.0)
        pool.append((s.frame1, s.frame2))
    srv = serve.Server(gp, 128, 96, hbm_budget_bytes=4 * serve.slot_bytes(gp, 128, 96) + (64 << 20), max_slots=3)
    assert len(srv.slots) == 3
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
