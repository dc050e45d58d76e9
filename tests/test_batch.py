"""Batched form: seeded workload recipes (CPU), and on the GPU the multi-stream,
graph-captured runner -- every pair's result is bitwise the one a plain
single-context run gives."""
import numpy as np
import pytest

from paper_1804_03787_gb300 import batch, scene


def test_batch_specs_are_seeded_and_in_range():
    a = batch.batch_specs(64, seed=3)
    b = batch.batch_specs(64, seed=3)
    assert a == b
    assert {(s["width"], s["height"]) for s in a} <= set(batch.BATCH_SIZES)
    assert all(3 <= s["n_layers"] <= 8 and s["max_disp"] == 96.0 for s in a)
    # all four sizes show up in a 64-pair draw
    assert len({(s["width"], s["height"]) for s in a}) == 4


def test_make_scenes_parallel_matches_serial():
    specs = batch.batch_specs(3, seed=1, sizes=((48, 40), (64, 48)))
    ser = batch.make_scenes(specs, workers=1)
    par = batch.make_scenes(specs, workers=3)
    for x, y in zip(ser, par):
        np.testing.assert_array_equal(x.frame1, y.frame1)
        np.testing.assert_array_equal(x.flow, y.flow)


def test_epe_of_identical_flows_is_zero():
    f = np.random.default_rng(0).normal(size=(5, 7, 2)).astype(np.float32)
    assert batch.epe(f, f) == 0.0
    assert abs(batch.epe(f + np.array([3.0, 4.0], np.float32), f) - 5.0) < 1e-6


@pytest.mark.gpu
def test_batched_runner_equals_plain_runs():
    import torch
    from paper_1804_03787_gb300 import gpm
    assert torch.cuda.is_available()
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=64)
    sizes = [(96, 72), (64, 48), (80, 64), (112, 80), (64, 64), (96, 48)]
    frames, ids = [], []
    for k, (w, h) in enumerate(sizes):
        s = scene.make_scene(w, h, seed=70 + k, n_layers=2, max_disp=5.0)
        frames.append((s.frame1, s.frame2))
        ids.append(500 + k)
    plain = []
    for (f1, f2), pid in zip(frames, ids):
        ctx = gpm.Context(gp, f1.shape[1], f1.shape[0])
        fl, oc = ctx.run([(torch.from_numpy(f1).cuda(), torch.from_numpy(f2).cuda())], pair_ids=[pid])
        plain.append((fl[0].cpu().numpy(), oc[0].cpu().numpy()))
        ctx.close()
    for streams, graph in ((1, False), (3, True)):
        r = batch.BatchRunner(gp, frames, ids, streams=streams, graph=graph)
        for _ in range(2):  # replaying the graph gives the same result again
            r.run()
            out = r.results()
            for k in range(len(frames)):
                np.testing.assert_array_equal(out[k][0], plain[k][0])
                np.testing.assert_array_equal(out[k][1], plain[k][1])
        r.close()


@pytest.mark.gpu
def test_one_launch_per_stage_covers_every_pair():
    """The pair index lives on the device: a call on six pairs of different sizes makes as many kernel launches
    as a call on one pair (every stage's launch covers up to eight pairs, blockIdx.z = pair), and each pair's
    result is bitwise that of the pair alone; the whole six-pair pipeline replays from one CUDA graph."""
    import torch
    from paper_1804_03787_gb300 import gpm
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=64)
    sizes = [(96, 72), (64, 48), (80, 64), (112, 80), (64, 64), (96, 48)]
    dev, ids = [], []
    for k, (w, h) in enumerate(sizes):
        s = scene.make_scene(w, h, seed=90 + k, n_layers=2, max_disp=5.0)
        dev.append((torch.from_numpy(s.frame1).cuda(), torch.from_numpy(s.frame2).cuda()))
        ids.append(700 + k)
    alone, counts = [], []
    for (f1, f2), pid in zip(dev, ids):
        ctx = gpm.Context(gp, 112, 80)
        fl, oc = ctx.run([(f1, f2)], pair_ids=[pid])
        torch.cuda.synchronize()
        alone.append((fl[0].cpu().numpy(), oc[0].cpu().numpy()))
        counts.append(ctx.launch_count())
        ctx.close()
    assert len(set(counts)) == 1
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ctx = gpm.Context(gp, 112, 80, max_pairs=len(dev), stream=st)
        flows = [torch.empty((f1.shape[0], f1.shape[1], 2), dtype=torch.float32, device="cuda") for f1, _ in dev]
        occs = [torch.empty((f1.shape[0], f1.shape[1]), dtype=torch.uint8, device="cuda") for f1, _ in dev]

        def run():
            ctx.match(dev, 0, pair_ids=ids)
            for level in range(1, gp.num_scales + 1):
                ctx.fit_planes(level)
                ctx.match(None, level)
            ctx.flow_and_occlusion(flows, occs)

        run()
    st.synchronize()
    assert ctx.launch_count() == counts[0]
    for k in range(len(dev)):
        np.testing.assert_array_equal(flows[k].cpu().numpy(), alone[k][0])
        np.testing.assert_array_equal(occs[k].cpu().numpy(), alone[k][1])
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        run()
    for f in flows:
        f.zero_()
    g.replay()
    torch.cuda.synchronize()
    for k in range(len(dev)):
        np.testing.assert_array_equal(flows[k].cpu().numpy(), alone[k][0])
    ctx.close()


def test_launch_shape_copy_and_autotune_cache():
    """with_launch_shape copies the parameters (the original is unchanged); the autotuner answers a batch shape
    it has seen from its cache, keyed by the frame sizes, patch radius and storage type, without timing."""
    from paper_1804_03787_gb300 import gpm
    gp = gpm.Params()
    gp.patch_radius = 4
    gp.storage = 0
    q = batch.with_launch_shape(gp, 16)
    assert q.sweep_blocks_per_sm == 16 and gp.sweep_blocks_per_sm == 0 and q.patch_radius == 4
    frames = [(np.zeros((48, 64, 3), np.float32), None), (np.zeros((40, 32, 3), np.float32), None)]
    cache = {(((32, 40), (64, 48)), 4, 0): ((2, 8), {(2, 8): 0.1})}
    assert batch.autotune(gp, frames, [0, 1], cache=cache) == ((2, 8), {(2, 8): 0.1})
