"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Bars (from the method's tolerances): integer NNF offsets, labels and
occlusion bits bit-exact except where the oracle logged a near tie
(|a - b| < 1e-5 relative at a decision) upstream; patch costs within 1e-5
relative; homographies within 1e-6 after normalisation; plane flows within
1e-5 px.  Lock-step tests feed the oracle's own state into the GPU (never the
other way) so that one near tie does not cascade.
"""
import numpy as np
import pytest

import oracle as O
from paper_1804_03787_gb300 import gpm, scene

from _parity import end_to_end_stats, COLOUR_ATOL, TIE, dilate, norm_h, oracle_frames, oracle_params, rel_close
from _parity import ransac_equal as _ransac_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    gpm.load()
    return t


def _scene(W, H, seed, layers=2, disp=5.0):
    return scene.make_scene(W, H, seed=seed, n_layers=layers, max_disp=disp, affine=True)


def _ctx(torch, gp, W, H, pairs=1):
    return gpm.Context(gp, W, H, pairs)


def _dev(torch, s):
    return torch.from_numpy(s.frame1).cuda(), torch.from_numpy(s.frame2).cuda()


CASES = [(64, 48, 2, (16, 8)), (70, 45, 3, (16, 8)), (66, 50, 1, (16, 8))]   # r = 1: a single 32-tap chunk


# ---------------------------------------------------------------- ingest and init
@pytest.mark.parametrize("W,H,r,cells", CASES)
def test_ingest_and_init_exact(torch, W, H, r, cells):
    s = _scene(W, H, seed=W)
    gp = gpm.default_params(patch_radius=r, cells=cells, pm_iters=0, num_hyp=64, seed=1234567890123)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)], pair_ids=[7])
    P = oracle_params(gp, W, H, pair_id=7)
    frames, g = oracle_frames(P, s.frame1, s.frame2)
    fr = ctx.export(gpm.FRAMES)
    for d in range(2):
        want = frames[0][d]
        np.testing.assert_allclose(fr[d, ..., :3], want, rtol=1.2e-7, atol=1e-12)
    nnf, cost = ctx.export(gpm.NNF), ctx.export(gpm.COST)
    for d in range(2):
        vx, vy, c = O.pm_init(P, frames[d][0], frames[d][1], d)
        np.testing.assert_array_equal(nnf[d, :, 0], vx)
        np.testing.assert_array_equal(nnf[d, :, 1], vy)
        assert rel_close(cost[d], c).all(), np.abs(cost[d] - c).max()
    ctx.close()


# ---------------------------------------------------------------- level-0 PatchMatch
def _oracle_pm(P, frames, d, level=0, mh=None, mi=None, frozen=None, state=None):
    """Oracle sweeps half-step by half-step with the near-tie log; returns
    (vx, vy, cost, cone) where cone holds every pixel a logged near tie may reach."""
    W, H = P.width, P.height
    if state is None:
        vx, vy, c = O.pm_init(P, frames[d][0], frames[d][1], d)
    else:
        vx, vy, c = (a.copy() for a in state)
    nh = 2 * P.pm_iters
    cone = np.zeros((H, W), bool)
    k = 0
    for it in range(P.pm_iters):
        for ph in range(2):
            amb = np.full(W * H, np.inf)
            O.pm_sweep(P, frames[d][0], frames[d][1], d, level, it, ph, mh, mi, frozen, vx, vy, c, amb)
            cone |= dilate((amb < TIE).reshape(H, W), nh - 1 - k)
            k += 1
    return vx, vy, c, cone


@pytest.mark.parametrize("W,H,r,cells", CASES)
def test_level0_patchmatch_matches_oracle_up_to_near_ties(torch, W, H, r, cells):
    s = _scene(W, H, seed=W + 1)
    gp = gpm.default_params(patch_radius=r, cells=cells, pm_iters=3, num_hyp=64)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    nnf, cost = ctx.export(gpm.NNF), ctx.export(gpm.COST)
    P = oracle_params(gp, W, H)
    frames, _ = oracle_frames(P, s.frame1, s.frame2)
    for d in range(2):
        vx, vy, c, cone = _oracle_pm(P, frames, d)
        diff = ((nnf[d, :, 0] != vx) | (nnf[d, :, 1] != vy)).reshape(H, W)
        assert not (diff & ~cone).any(), f"dir {d}: {int((diff & ~cone).sum())} unexplained NNF differences"
        assert diff.mean() < 0.01
        same = ~diff.reshape(-1)
        assert rel_close(cost[d][same], c[same]).all()
    ctx.close()


@pytest.mark.parametrize("W,H,r", [(4, 4, 4), (5, 7, 1), (9, 4, 4), (37, 5, 2), (33, 9, 3)])
def test_level0_patchmatch_tiny_ragged_frames(torch, W, H, r):
    """Level 0 alone (no plane levels) on frames smaller than one sweep tile (32 x 8 pixels) in either axis or
    both, some smaller than the patch: the tile's partial rows and columns, clamped taps, no patch-sum bound
    (no pixel's patch fits in the frame) or only a few interior pixels.  Same bars as the larger cases."""
    s = _scene(W, H, seed=W * 7 + H)
    gp = gpm.default_params(patch_radius=r, cells=(), pm_iters=4, num_hyp=64)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    nnf, cost = ctx.export(gpm.NNF), ctx.export(gpm.COST)
    P = oracle_params(gp, W, H)
    frames, _ = oracle_frames(P, s.frame1, s.frame2)
    diffs = []
    for d in range(2):
        vx, vy, c, cone = _oracle_pm(P, frames, d)
        diff = ((nnf[d, :, 0] != vx) | (nnf[d, :, 1] != vy)).reshape(H, W)
        assert not (diff & ~cone).any(), f"dir {d}: {int((diff & ~cone).sum())} unexplained NNF differences"
        same = ~diff.reshape(-1)
        assert rel_close(cost[d][same], c[same]).all()
        diffs.append(diff)
    # the final map without plane levels (Sec. 3.4.1): no pixel has a plane, so the flow is the NNF offset and
    # every pixel is occluded
    flows, occs = ctx.flow_and_occlusion()
    torch.cuda.synchronize()
    R = O.run(P, s.frame1, s.frame2)
    gf, of = flows[0].cpu().numpy(), R.flow[0].reshape(H, W, 2)
    np.testing.assert_array_equal(gf[~diffs[0]], of[~diffs[0]])
    np.testing.assert_array_equal(occs[0].cpu().numpy().reshape(-1), np.asarray(R.occ[0]).reshape(-1))
    ctx.close()


# ---------------------------------------------------------------- one level of Algorithm 1, lock-step
def _oracle_level(P, frames, l, vx, vy, mh, mi, acc, cue):
    """One level of the oracle, stage by stage, with the per-pixel near-tie logs."""
    n = P.width * P.height
    T, S1, C, amb = [], [], [], []
    for d in range(2):
        O.fit_level(P, frames[d][0], frames[d][1], d, l, 1, vx[d], vy[d], None, mh[d], mi[d])
    for d in range(2):
        t = O.Labels.empty(n, P.eps)
        a = np.zeros(n, np.uint8)
        O.assign(P, frames[d][0], frames[d][1], l, 1, mh[d], mi[d], None, t, a)
        T.append(t)
        amb.append(a)
    for d in range(2):
        O.cue_counts(P, l, 1, T[d], T[1 - d], mi[d], amb[d])
    for d in range(2):
        O.cue_invalidate(P, l, 1, mi[d])
    resid = []
    for d in range(2):
        t = O.Labels.empty(n, P.eps)
        O.assign(P, frames[d][0], frames[d][1], l, 1, mh[d], mi[d], None, t, amb[d])
        S1.append(t)
        resid.append((t.m < 0).astype(np.uint8))
    for d in range(2):
        O.fit_level(P, frames[d][0], frames[d][1], d, l, 2, vx[d], vy[d], resid[d], mh[d], mi[d])
    for d in range(2):
        c = S1[d].copy()
        O.assign(P, frames[d][0], frames[d][1], l, 2, mh[d], mi[d], resid[d], c, amb[d])
        C.append(c)
    for d in range(2):
        O.cue_counts(P, l, 2, C[d], C[1 - d], mi[d], amb[d])
    for d in range(2):
        O.cue_invalidate(P, l, 2, mi[d])
    for d in range(2):
        c = S1[d].copy()
        O.assign(P, frames[d][0], frames[d][1], l, 2, mh[d], mi[d], resid[d], c, amb[d])
        C[d] = c
    frozen = []
    for d in range(2):
        O.many_to_one(P, C[d], cue[d], amb[d])
        O.merge(P, C[d], acc[d], amb[d])
        f = np.zeros(n, np.uint8)
        O.nnf_update(P, acc[d], vx[d], vy[d], f)
        frozen.append(f)
    return S1, C, frozen, amb


CUE_FIELDS = [O.MI_VALID, O.MI_NASSIGN, O.MI_NSYM]


def _label_report(bad, g, o, d, W, k=8):
    """(x, y, GPU model, oracle model, GPU L, oracle L, GPU flow, oracle flow) of the first k flagged pixels."""
    out = []
    for i in np.flatnonzero(bad.reshape(-1))[:k]:
        out.append((int(i % W), int(i // W), int(g[0][d][i]), int(o.m[i]), float(g[1][d][i]), float(o.L[i]),
                    tuple(np.round(g[2][d][i], 6)), (round(float(o.fx[i]), 6), round(float(o.fy[i]), 6))))
    return out


def _cues_equal(gmi, omi, ids):
    return np.array([all(gmi[m][f] == omi[m][f] for f in CUE_FIELDS) for m in ids])


def _window_box(P, cells, c, margin):
    gx, gy = O.grid_axis(P.width, cells[0]), O.grid_axis(P.height, cells[0])
    x0, y0 = gx[c % len(gx)], gy[c // len(gx)]
    return slice(max(0, y0 - margin), y0 + cells[0] + margin), slice(max(0, x0 - margin), x0 + cells[0] + margin)


@pytest.mark.parametrize("W,H,r,cells", CASES)
def test_fit_planes_level1_lockstep(torch, W, H, r, cells):
    """One level of Algorithm 1 from the oracle's level-0 NNF.

    RANSAC outputs must match for every window whose fit the oracle did not
    flag as a near tie.  Cue counts (pixels assigned / symmetric) read the
    tentative labels of both directions: they may differ only in windows that
    hold a pixel with a logged near tie (within the motion margin), and labels
    only on such pixels or in windows whose model differs."""
    s = _scene(W, H, seed=W + 2)
    gp = gpm.default_params(patch_radius=r, cells=cells, pm_iters=3, num_hyp=96)
    P = oracle_params(gp, W, H)
    frames, _ = oracle_frames(P, s.frame1, s.frame2)
    R0 = O.run(P, s.frame1, s.frame2, stop_after=0)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    nnf0 = np.stack([np.stack([R0.vx[d], R0.vy[d]], 1) for d in range(2)]).astype(np.int32)
    ctx.import_state(gpm.NNF, nnf0, level=0)
    ctx.fit_planes(1)
    gmh, gmi = ctx.export(gpm.MODELS), ctx.export(gpm.MODEL_INFO)
    gs1 = ctx.export(gpm.STAGE1_LABELS)
    glv = ctx.export(gpm.LEVEL_LABELS)
    gacc = ctx.export(gpm.LABELS)
    gcue = ctx.export(gpm.CUES)
    gnnf = ctx.export(gpm.NNF)
    n = W * H
    vx = [R0.vx[d].copy() for d in range(2)]
    vy = [R0.vy[d].copy() for d in range(2)]
    mh = [np.zeros_like(R0.mh[d]) for d in range(2)]
    mi = [np.zeros_like(R0.mi[d]) for d in range(2)]
    acc = [O.Labels.empty(n, P.eps) for _ in range(2)]
    cue = [np.zeros(n, np.uint8) for _ in range(2)]
    S1, C, frozen, amb = _oracle_level(P, frames, 1, vx, vy, mh, mi, acc, cue)
    ncell = int(O.cell_base(P)[1])
    margin = 8   # motion bound of the scene plus rounding
    ids = np.arange(2 * ncell)
    first = ids[::2]
    okr = [_ransac_equal(gmh[d], gmi[d], mh[d], mi[d], ids) for d in range(2)]
    # pixels near a window whose fit differs in either direction, or near a logged near tie:
    # the symmetry cue of one direction reads the labels of the other
    upstream = (amb[0] | amb[1]).reshape(H, W).astype(bool)
    for d in range(2):
        for m in ids[~okr[d]]:
            ys, xs = _window_box(P, cells, m // 2, margin)
            upstream[ys, xs] = True
    for d in range(2):
        oracle_tie = (mi[d][ids, O.MI_FLAGS] & O.F_AMBIG) > 0
        # stage-1 fits see identical inputs: only oracle-flagged near ties may differ
        bad1 = first[~okr[d][first] & ~oracle_tie[first]]
        assert len(bad1) == 0, f"dir {d}: stage-1 RANSAC differs in windows {bad1 // 2}"
        # cue counts: explained by an upstream difference near the window
        okc = _cues_equal(gmi[d], mi[d], ids)
        expl_w = np.zeros(2 * ncell, bool)
        for m in ids:
            ys, xs = _window_box(P, cells, m // 2, margin)
            expl_w[m] = upstream[ys, xs].any() or oracle_tie[m]
        bad_c = ids[~okc & ~expl_w & okr[d]]
        assert len(bad_c) == 0, f"dir {d}: cue counts differ without a near tie in models {bad_c}"
        # labels: differences on near-tie pixels or inside windows whose model differs
        expl = amb[d].reshape(H, W).astype(bool)
        model_ok = okr[d] & okc
        for m in ids[~model_ok]:
            ys, xs = _window_box(P, cells, m // 2, 0)
            expl[ys, xs] = True
        # a many-to-one loss is decided by the lowest (L, index) claimant of the target, and claimants of one
        # target lie within the motion bound of each other: a loss may differ near an explained pixel
        lost = (((gcue[d] | cue[d]) & O.CUE_M2O) > 0).reshape(H, W)
        expl |= dilate(expl, margin) & lost
        for name, g, o in (("stage-1", gs1, S1[d]), ("level", glv, C[d])):
            diff = (g[0][d] != o.m).reshape(H, W)
            assert not (diff & ~expl).any(), (f"dir {d} {name} labels: {int((diff & ~expl).sum())} unexplained",
                                              _label_report(diff & ~expl, g, o, d, W))
            assert diff.mean() < 0.05
            # flows and losses where both sides chose the same, identical model
            same = (~diff.reshape(-1)) & (o.m >= 0)
            same[same] &= model_ok[o.m[same]]
            flo = np.stack([o.fx, o.fy], 1)
            assert np.abs(g[2][d][same] - flo[same]).max(initial=0) < 1e-5
            assert rel_close(g[1][d][same], o.L[same], atol=COLOUR_ATOL).all()
        diff = (gacc[0][d] != acc[d].m) | (gcue[d] != cue[d])
        assert not (diff.reshape(H, W) & ~expl).any()
        nd = ((gnnf[d, :, 0] != vx[d]) | (gnnf[d, :, 1] != vy[d])).reshape(H, W)
        assert not (nd & ~expl).any()
    ctx.close()


# ---------------------------------------------------------------- restricted, plane-distorted PatchMatch
@pytest.mark.parametrize("W,H,r,cells", CASES)
def test_restricted_patchmatch_level1_lockstep(torch, W, H, r, cells):
    """Sec. 3.3.2 from the oracle's state after its level-1 fit (planes, merged
    labels, updated NNF imported): unassigned pixels only, patches distorted by
    the home-window plane, plane candidates; near-tie cone rule as at level 0."""
    s = _scene(W, H, seed=11 + W, disp=6.0)
    gp = gpm.default_params(patch_radius=r, cells=cells, pm_iters=2, num_hyp=96)
    P = oracle_params(gp, W, H)
    frames, _ = oracle_frames(P, s.frame1, s.frame2)
    R0 = O.run(P, s.frame1, s.frame2, stop_after=0)
    R1 = O.run(P, s.frame1, s.frame2, stop_after=1)
    n = W * H
    vx = [R0.vx[d].copy() for d in range(2)]
    vy = [R0.vy[d].copy() for d in range(2)]
    mh = [np.zeros_like(R0.mh[d]) for d in range(2)]
    mi = [np.zeros_like(R0.mi[d]) for d in range(2)]
    acc = [O.Labels.empty(n, P.eps) for _ in range(2)]
    cue = [np.zeros(n, np.uint8) for _ in range(2)]
    S1, C, frozen, amb = _oracle_level(P, frames, 1, vx, vy, mh, mi, acc, cue)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    ctx.import_state(gpm.NNF, np.stack([np.stack([vx[d], vy[d]], 1) for d in range(2)]).astype(np.int32), 1,
                     after_fit=True)
    ctx.import_state(gpm.MODELS, np.stack(mh), 1, after_fit=True)
    ctx.import_state(gpm.MODEL_INFO, np.stack(mi), 1, after_fit=True)
    ctx.import_state(gpm.LABELS, (np.stack([acc[d].m for d in range(2)]),
                                  np.stack([acc[d].L for d in range(2)]).astype(np.float32),
                                  np.stack([np.stack([acc[d].fx, acc[d].fy], 1) for d in range(2)])), 1,
                     after_fit=True)
    ctx.import_state(gpm.CUES, np.stack(cue), 1, after_fit=True)
    ctx.match(None, 1)
    gnnf, gcost = ctx.export(gpm.NNF), ctx.export(gpm.COST)
    for d in range(2):
        cost = np.zeros(n)
        O.pm_recost(P, frames[d][0], frames[d][1], 1, mh[d], mi[d], frozen[d], vx[d], vy[d], cost)
        ox, oy, oc, cone = _oracle_pm(P, frames, d, level=1, mh=mh[d], mi=mi[d], frozen=frozen[d],
                                      state=(vx[d], vy[d], cost))
        np.testing.assert_array_equal(ox, R1.vx[d])   # the stage-by-stage oracle equals its own pipeline
        diff = ((gnnf[d, :, 0] != ox) | (gnnf[d, :, 1] != oy)).reshape(H, W)
        assert not (diff & ~cone).any(), int((diff & ~cone).sum())
        upd = (frozen[d] == 0) & ~diff.reshape(-1)
        assert upd.sum() > 0
        assert rel_close(gcost[d][upd], oc[upd]).all()
    ctx.close()


# ---------------------------------------------------------------- fill and final map, lock-step
@pytest.mark.parametrize("W,H,r,cells", CASES)
def test_fill_and_final_lockstep(torch, W, H, r, cells):
    s = _scene(W, H, seed=W + 3)
    gp = gpm.default_params(patch_radius=r, cells=cells, pm_iters=2, num_hyp=64, fill_iters=5)
    P = oracle_params(gp, W, H)
    frames, _ = oracle_frames(P, s.frame1, s.frame2)
    L = len(cells)
    R = O.run(P, s.frame1, s.frame2, stop_after=L)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    n = W * H
    ctx.import_state(gpm.NNF, np.stack([np.stack([R.vx[d], R.vy[d]], 1) for d in range(2)]).astype(np.int32), L)
    ctx.import_state(gpm.MODELS, np.stack(R.mh), L)
    ctx.import_state(gpm.MODEL_INFO, np.stack(R.mi), L)
    ctx.import_state(gpm.LABELS, (np.stack([R.acc[d].m for d in range(2)]),
                                  np.stack([R.acc[d].L for d in range(2)]).astype(np.float32),
                                  np.stack([np.stack([R.acc[d].fx, R.acc[d].fy], 1) for d in range(2)])), L)
    ctx.import_state(gpm.CUES, np.stack(R.cue), L)
    flows, occs = ctx.flow_and_occlusion()
    torch.cuda.synchronize()
    gflow, gocc = flows[0].cpu().numpy().reshape(n, 2), occs[0].cpu().numpy().reshape(n)
    acc = R.acc[0].copy()
    amb = np.zeros(n, np.uint8)
    O.fill(P, frames[0][0], frames[0][1], R.mh[0], R.mi[0], R.cue[0], acc, amb)
    oflow, oocc = O.final(P, frames[0][0], frames[0][1], acc, R.vx[0], R.vy[0], R.cue[0], amb)
    # Sec. 3.4.1: occlusion bits and flows equal except at the near ties the oracle logs (fill choices and
    # occlusion decisions within the bands of their thresholds, or next to such a choice); flows within the FP32
    # mapping's error
    assert not ((gocc != oocc) & (amb == 0)).any(), int(((gocc != oocc) & (amb == 0)).sum())
    fd = np.hypot(*(gflow - oflow).T)
    tol = 1e-5 + 4 * 2.0 ** -24 * np.hypot(oflow[:, 0], oflow[:, 1])
    assert not ((fd > tol) & (amb == 0)).any(), int(((fd > tol) & (amb == 0)).sum())
    ctx.close()


# ---------------------------------------------------------------- whole method
def test_tiny_config_end_to_end(torch):
    """128x96, 2 layers, r=3, cells 32/16/8, 4 iterations, 256 hypotheses: the whole method against the oracle.
    Where both sides give a pixel the same plane, its final flow is that plane's mapping (Sec. 3.4.1): the flows
    agree within the FP32 mapping's error and their EPE against the ground truth within 1e-3 px.  Different plane
    choices come from near ties between overlapping windows' fits of one surface and are few.  Pixels without a
    plane keep their NNF offsets from the random search, where a near tie upstream changes an offset by many
    pixels; over the whole frame the EPE still agrees within 1e-3 px (the final-flow bar) and under 1 % of the
    flows differ.  Each stage on its own is checked against the oracle given the same state, with every
    difference at a logged near tie, by the lock-step tests above and the full-size tests."""
    s = scene.tiny_scene(0)
    gp = gpm.default_params()
    ctx = _ctx(torch, gp, 128, 96)
    f1, f2 = _dev(torch, s)
    flows, occs = ctx.run([(f1, f2)])
    torch.cuda.synchronize()
    gflow = flows[0].cpu().numpy()
    P = oracle_params(gp, 128, 96)
    R = O.run(P, s.frame1, s.frame2)
    oflow = R.flow[0].reshape(96, 128, 2)
    st = end_to_end_stats(ctx, R, gflow, oflow, s.flow, s.occ, 96, 128)
    print("tiny:", {k: round(v, 5) for k, v in st.items()})
    # the same plane decision: the flows agree within the FP32 mapping's error, the EPE within 1e-3 px
    assert st["same_share"] > 0.8 and st["same_max_flow_diff"] < 1e-3, st
    assert abs(st["epe_same_gpu"] - st["epe_same_oracle"]) <= 1e-3, st
    # different plane decisions (near ties between overlapping windows' fits of one surface) are few, and the
    # whole frame's EPE agrees within the final-flow bar, 1e-3 px
    assert st["label_agree"] > 0.99 and st["plane_agree"] > 0.99, st
    assert st["agree"] > 0.99 and abs(st["epe_gpu"] - st["epe_oracle"]) <= 1e-3, st
    # the occlusion map (Sec. 3.4.1): the same bits except where a plane decision differed upstream
    gocc = occs[0].cpu().numpy().reshape(-1)
    oocc = np.asarray(R.occ[0]).reshape(-1)
    occ_agree = float(np.mean(gocc == oocc))
    print(f"tiny: occlusion bits agree on {occ_agree:.5f}")
    assert occ_agree > 0.99, occ_agree
    ctx.close()


def test_repeatable_bitwise(torch):
    s = _scene(70, 45, seed=5)
    gp = gpm.default_params(patch_radius=3, cells=(16, 8), pm_iters=2, num_hyp=64)
    outs = []
    for _ in range(2):
        ctx = _ctx(torch, gp, 70, 45)
        flows, occs = ctx.run([_dev(torch, s)])
        outs.append((flows[0].cpu().numpy(), occs[0].cpu().numpy(), ctx.export(gpm.MODELS)))
        ctx.close()
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------- reduced-precision storage
def _quantise(a, kind):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32))
    return (t.to(torch.float16 if kind == "f16" else torch.bfloat16).to(torch.float32)).numpy()


@pytest.mark.parametrize("kind,storage", [("f16", gpm.GPM_F16), ("bf16", gpm.GPM_BF16)])
def test_reduced_precision_storage(torch, kind, storage):
    """Frames stored as FP16/BF16 texels, FP32 arithmetic: against the oracle run
    on the dequantised frames the level-0 NNF follows the near-tie rule; against
    the oracle on the original frames the error is reported and bounded."""
    W, H, r, cells = 64, 48, 2, (16, 8)
    s = _scene(W, H, seed=21)
    gp = gpm.default_params(patch_radius=r, cells=cells, pm_iters=3, num_hyp=64, storage=storage)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    nnf, cost = ctx.export(gpm.NNF), ctx.export(gpm.COST)
    fr = ctx.export(gpm.FRAMES)
    P = oracle_params(gp, W, H)
    frames32, g = oracle_frames(P, s.frame1, s.frame2)
    # the GPU stores round(I1) and round(gain * I2): the oracle sees exactly those values
    q1 = _quantise(s.frame1, kind).astype(np.float64)
    q2 = _quantise((s.frame2.astype(np.float64) * g).astype(np.float32), kind).astype(np.float64)
    np.testing.assert_array_equal(fr[0, ..., :3], q1)
    np.testing.assert_array_equal(fr[1, ..., :3], q2)
    Pq = oracle_params(gp, W, H)
    Pq.gain_normalize = 0
    framesq = [(q1, q2), (q2, q1)]
    agree = []
    for d in range(2):
        vx, vy, c, cone = _oracle_pm(Pq, framesq, d)
        diff = ((nnf[d, :, 0] != vx) | (nnf[d, :, 1] != vy)).reshape(H, W)
        assert not (diff & ~cone).any()
        same = ~diff.reshape(-1)
        assert rel_close(cost[d][same], c[same]).all()
        # against the FP64 oracle on the original frames
        vx0, vy0, c0, _ = _oracle_pm(P, frames32, d)
        agree.append(np.mean((nnf[d, :, 0] == vx0) & (nnf[d, :, 1] == vy0)))
    print(f"{kind}: level-0 NNF agreement with the FP64 oracle on FP32 frames {np.mean(agree):.4f}")
    assert np.mean(agree) > 0.8
    ctx.close()


@pytest.mark.parametrize("kind,storage", [("f16", gpm.GPM_F16), ("bf16", gpm.GPM_BF16)])
def test_reduced_precision_end_to_end(torch, kind, storage):
    """Tiny config, frames stored as FP16/BF16: the whole method against the oracle on the dequantised frames
    (FP16: the bars of the FP32 end-to-end test; BF16: see below), and the accuracy change against the FP64 oracle
    on the original frames reported and loosely bounded."""
    s = scene.tiny_scene(0)
    gp = gpm.default_params(storage=storage)
    ctx = _ctx(torch, gp, 128, 96)
    flows, occs = ctx.run([_dev(torch, s)])
    torch.cuda.synchronize()
    gflow = flows[0].cpu().numpy()
    P = oracle_params(gp, 128, 96)
    _, g = oracle_frames(P, s.frame1, s.frame2)
    q1 = _quantise(s.frame1, kind).astype(np.float64)
    q2 = _quantise((s.frame2.astype(np.float64) * g).astype(np.float32), kind).astype(np.float64)
    Pq = oracle_params(gp, 128, 96)
    Pq.gain_normalize = 0
    Rq = O.run(Pq, q1, q2)
    qflow = Rq.flow[0].reshape(96, 128, 2)
    vis = s.occ == 0
    agree = np.mean(np.hypot(*(gflow - qflow).transpose(2, 0, 1)) < 1e-4)
    epe_g = np.hypot(*(gflow - s.flow).transpose(2, 0, 1))[vis].mean()
    epe_q = np.hypot(*(qflow - s.flow).transpose(2, 0, 1))[vis].mean()
    R = O.run(P, s.frame1, s.frame2)
    epe_o = np.hypot(*(R.flow[0].reshape(96, 128, 2) - s.flow).transpose(2, 0, 1))[vis].mean()
    print(f"{kind}: flow agreement with the oracle on dequantised frames {agree:.4f}; EPE nocc gpu {epe_g:.4f}, "
          f"oracle (dequantised) {epe_q:.4f}, oracle (FP64 frames) {epe_o:.4f}")
    # FP16 holds the FP32 end-to-end bars.  BF16's 8-bit mantissas make many candidates' costs exactly equal sums
    # of equal texels; FP32 and FP64 then round those sums differently and break the ties apart (measured: flow
    # agreement 0.976, EPE 1.1e-3 apart).
    assert agree > (0.99 if kind == "f16" else 0.97)
    assert abs(epe_g - epe_q) <= (1e-3 if kind == "f16" else 2e-3)
    # the accuracy change against the FP64 oracle on the original frames: reported, and bounded only loosely
    assert abs(epe_g - epe_o) < 0.1
    ctx.close()


def test_frame_dtypes_per_pair(torch):
    """Frames given as FP16 or BF16 (per pair, through gpm_pair.dtype) are converted exactly on ingest: the whole
    method gives bitwise the results of the FP32 frames holding the same values, alone and with pairs of other
    dtypes in the same call."""
    s = scene.tiny_scene(0)
    gp = gpm.default_params()
    H, W = s.frame1.shape[:2]
    ctx = _ctx(torch, gp, W, H, pairs=3)
    ins = {}
    for dt in (torch.float16, torch.bfloat16):
        a = torch.from_numpy(s.frame1).cuda().to(dt)
        b = torch.from_numpy(s.frame2).cuda().to(dt)
        ins[dt] = ((a, b), (a.float(), b.float()))
    ref = {}
    for dt, (low, f32) in ins.items():
        for form, fr in (("low", low), ("f32", f32)):
            flows, occs = ctx.run([fr], pair_ids=[5])
            torch.cuda.synchronize()
            ref[(dt, form)] = (flows[0].cpu().numpy(), occs[0].cpu().numpy(), ctx.export(gpm.NNF)[0].copy())
        for k in range(3):
            np.testing.assert_array_equal(ref[(dt, "low")][k], ref[(dt, "f32")][k])
    # one call: FP32, FP16 and BF16 pairs together, each as alone
    f32 = (torch.from_numpy(s.frame1).cuda(), torch.from_numpy(s.frame2).cuda())
    flows, occs = ctx.run([ins[torch.float16][0], f32, ins[torch.bfloat16][0]], pair_ids=[5, 5, 5])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(flows[0].cpu().numpy(), ref[(torch.float16, "f32")][0])
    np.testing.assert_array_equal(flows[2].cpu().numpy(), ref[(torch.bfloat16, "f32")][0])
    np.testing.assert_array_equal(occs[2].cpu().numpy(), ref[(torch.bfloat16, "f32")][1])
    ctx.close()


# ---------------------------------------------------------------- HSV histogram equalisation (Sec. 4.2)
def test_equalized_ingest_matches_oracle(torch):
    """Ingest with equalize=1: both stored frames against the oracle's FP64 equalisation (then gain). The GPU
    rescales RGB by V'/V in FP32, the oracle goes through HSV and back in FP64: a few float roundings apart."""
    W, H = 70, 45
    s = _scene(W, H, seed=31)
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=0, num_hyp=32, equalize=1)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    fr = ctx.export(gpm.FRAMES)
    P = oracle_params(gp, W, H)
    e1 = O.hsv_equalize(P, s.frame1)
    e2 = O.hsv_equalize(P, s.frame2)
    g = O.gain(P, e1, e2)
    np.testing.assert_allclose(fr[0, ..., :3], e1, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(fr[1, ..., :3], e2 * g, rtol=1e-6, atol=1e-7)
    # equalisation changed the frames (the scenes do not fill [0, 1] evenly)
    assert np.abs(e1 - s.frame1).max() > 0.05
    ctx.close()


def test_equalized_tiny_end_to_end(torch):
    """Tiny config with equalize=1 against the oracle with equalize=1: the bars of the plain end-to-end test."""
    s = scene.tiny_scene(0)
    gp = gpm.default_params(equalize=1)
    ctx = _ctx(torch, gp, 128, 96)
    flows, occs = ctx.run([_dev(torch, s)])
    torch.cuda.synchronize()
    gflow = flows[0].cpu().numpy()
    P = oracle_params(gp, 128, 96)
    assert P.equalize == 1
    R = O.run(P, s.frame1, s.frame2)
    oflow = R.flow[0].reshape(96, 128, 2)
    vis = s.occ == 0
    agree = np.mean(np.hypot(*(gflow - oflow).transpose(2, 0, 1)) < 1e-4)
    epe_g = np.hypot(*(gflow - s.flow).transpose(2, 0, 1))[vis].mean()
    epe_o = np.hypot(*(oflow - s.flow).transpose(2, 0, 1))[vis].mean()
    print(f"equalized tiny: flow agreement {agree:.4f}, EPE nocc gpu {epe_g:.4f} oracle {epe_o:.4f}")
    assert agree > 0.95
    assert abs(epe_g - epe_o) < 0.01
    ctx.close()


# ---------------------------------------------------------------- large windows (the paper's preset sizes)
@pytest.mark.parametrize("W,H,cells", [(192, 112, (80, 40)), (288, 192, (96, 48))])
def test_large_windows_end_to_end(torch, W, H, cells):
    """Windows of 80 and 40 px (the paper's radius-40/20 windows, 2 levels, 7x7 patches) on a 192x112 pair, and
    the largest windows the library takes (96 px: 9,216 matches, 144 KiB of shared memory in RANSAC, the widest
    128-bit hypothesis bounds) on a 288x192 pair: the whole method against the oracle, with the bars of the tiny
    end-to-end test."""
    s = scene.make_scene(W, H, seed=9, n_layers=2, max_disp=6.0, affine=True)
    gp = gpm.default_params(patch_radius=3, cells=cells, pm_iters=4, num_hyp=128)
    ctx = _ctx(torch, gp, W, H)
    flows, _ = ctx.run([_dev(torch, s)])
    torch.cuda.synchronize()
    gflow = flows[0].cpu().numpy()
    R = O.run(oracle_params(gp, W, H), s.frame1, s.frame2)
    oflow = R.flow[0].reshape(H, W, 2)
    vis = s.occ == 0
    agree = np.mean(np.hypot(*(gflow - oflow).transpose(2, 0, 1)) < 1e-4)
    epe_g = np.hypot(*(gflow - s.flow).transpose(2, 0, 1))[vis].mean()
    epe_o = np.hypot(*(oflow - s.flow).transpose(2, 0, 1))[vis].mean()
    print(f"{cells} windows: flow agreement {agree:.4f}, EPE nocc gpu {epe_g:.4f} oracle {epe_o:.4f}")
    assert agree > 0.95
    assert abs(epe_g - epe_o) < 0.01
    ctx.close()


# ---------------------------------------------------------------- census data term (Sec. 6)
@pytest.mark.parametrize("W,H,r", [(64, 48, 2), (70, 45, 3)])
def test_census_level0_equals_oracle_exactly(torch, W, H, r):
    """Level-0 PatchMatch with the census data term: integer Hamming costs leave no near ties, so the NNF must
    equal the oracle's exactly (both directions) and the costs agree to the division."""
    s = _scene(W, H, seed=W + 5)
    gp = gpm.default_params(patch_radius=r, cells=(16, 8), pm_iters=3, num_hyp=32, census=1)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)], pair_ids=[3])
    nnf, cost = ctx.export(gpm.NNF), ctx.export(gpm.COST)
    R = O.run(oracle_params(gp, W, H, pair_id=3), s.frame1, s.frame2, stop_after=0)
    for d in range(2):
        np.testing.assert_array_equal(nnf[d, :, 0], R.vx[d])
        np.testing.assert_array_equal(nnf[d, :, 1], R.vy[d])
        np.testing.assert_allclose(cost[d], R.cost[d], rtol=1e-6, atol=0)
    ctx.close()


def test_census_tiny_end_to_end(torch):
    """Tiny config with the census data term against the oracle with it: the bars of the plain end-to-end test."""
    s = scene.tiny_scene(0)
    gp = gpm.default_params(census=1)
    ctx = _ctx(torch, gp, 128, 96)
    flows, _ = ctx.run([_dev(torch, s)])
    torch.cuda.synchronize()
    gflow = flows[0].cpu().numpy()
    R = O.run(oracle_params(gp, 128, 96), s.frame1, s.frame2)
    oflow = R.flow[0].reshape(96, 128, 2)
    vis = s.occ == 0
    agree = np.mean(np.hypot(*(gflow - oflow).transpose(2, 0, 1)) < 1e-4)
    epe_g = np.hypot(*(gflow - s.flow).transpose(2, 0, 1))[vis].mean()
    epe_o = np.hypot(*(oflow - s.flow).transpose(2, 0, 1))[vis].mean()
    print(f"census tiny: flow agreement {agree:.4f}, EPE nocc gpu {epe_g:.4f} oracle {epe_o:.4f}")
    assert agree > 0.95
    assert abs(epe_g - epe_o) < 0.01
    ctx.close()


# ---------------------------------------------------------------- edge-aware fill of unassigned pixels
@pytest.mark.parametrize("W,H,r,cells", CASES)
def test_interp_fill_lockstep(torch, W, H, r, cells):
    """The oracle's state before the final stage imported, interp=1: pixels without a plane take the geodesically
    nearest assigned pixel's plane.  Seeds are integer geodesics (the same on both sides for the same labels), so
    the filled flows agree up to the FP32 evaluation of the seed plane."""
    s = _scene(W, H, seed=W + 3)
    gp = gpm.default_params(patch_radius=r, cells=cells, pm_iters=2, num_hyp=64, fill_iters=5, interp=1)
    P = oracle_params(gp, W, H)
    frames, _ = oracle_frames(P, s.frame1, s.frame2)
    L = len(cells)
    R = O.run(P, s.frame1, s.frame2, stop_after=L)
    ctx = _ctx(torch, gp, W, H)
    ctx.match([_dev(torch, s)])
    n = W * H
    ctx.import_state(gpm.NNF, np.stack([np.stack([R.vx[d], R.vy[d]], 1) for d in range(2)]).astype(np.int32), L)
    ctx.import_state(gpm.MODELS, np.stack(R.mh), L)
    ctx.import_state(gpm.MODEL_INFO, np.stack(R.mi), L)
    ctx.import_state(gpm.LABELS, (np.stack([R.acc[d].m for d in range(2)]),
                                  np.stack([R.acc[d].L for d in range(2)]).astype(np.float32),
                                  np.stack([np.stack([R.acc[d].fx, R.acc[d].fy], 1) for d in range(2)])), L)
    ctx.import_state(gpm.CUES, np.stack(R.cue), L)
    flows, occs = ctx.flow_and_occlusion()
    torch.cuda.synchronize()
    gflow = flows[0].cpu().numpy().reshape(n, 2)
    acc = R.acc[0].copy()
    O.fill(P, frames[0][0], frames[0][1], R.mh[0], R.mi[0], R.cue[0], acc)
    oflow, _ = O.final(P, frames[0][0], frames[0][1], acc, R.vx[0], R.vy[0], R.cue[0])
    seed = O.interp_seeds(P, s.frame1, acc.m)
    O.interp_flow(P, R.mh[0], acc, seed, oflow)
    filled = (acc.m < 0) & (seed >= 0)
    assert filled.any()
    fd = np.hypot(*(gflow - oflow).T)
    assert np.mean(fd > 1e-5) < 0.005, np.mean(fd > 1e-5)
    assert np.mean(fd[filled] > 1e-3) < 0.02, np.mean(fd[filled] > 1e-3)
    ctx.close()


def test_interp_tiny_end_to_end(torch):
    """Tiny config with interp=1 against the oracle with it: the plain end-to-end bars, and the EPE over all
    pixels (occluded ones included) much lower than without the fill."""
    s = scene.tiny_scene(0)
    gp = gpm.default_params(interp=1)
    ctx = _ctx(torch, gp, 128, 96)
    flows, _ = ctx.run([_dev(torch, s)])
    torch.cuda.synchronize()
    gflow = flows[0].cpu().numpy()
    R = O.run(oracle_params(gp, 128, 96), s.frame1, s.frame2)
    oflow = R.flow[0].reshape(96, 128, 2)
    agree = np.mean(np.hypot(*(gflow - oflow).transpose(2, 0, 1)) < 1e-3)
    epe_all = np.hypot(*(gflow - s.flow).transpose(2, 0, 1)).mean()
    ctx0 = _ctx(torch, gpm.default_params(), 128, 96)
    f0, _ = ctx0.run([_dev(torch, s)])
    epe0 = np.hypot(*(f0[0].cpu().numpy() - s.flow).transpose(2, 0, 1)).mean()
    print(f"fill tiny: flow agreement {agree:.4f}, EPE all with fill {epe_all:.3f}, without {epe0:.3f}")
    assert agree > 0.95
    assert epe_all < epe0
    ctx.close()
    ctx0.close()
