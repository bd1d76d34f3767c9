"""Batched densification (persistent launch per phase, CUDA graph, autotuner).

Every keyframe of a batch runs the single-keyframe per-pixel computation, so
its maps must equal what pmsp_densify gives for it alone (compared bit for
bit, with a cost tolerance of 1e-6 as the only slack for the compiler's
instruction scheduling), and the oracle pins the values themselves.
"""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_16266_gb300 as pm
    return pm


@pytest.fixture(scope="module")
def ctx(pm):
    import torch
    c = pm.Context(0, stream=torch.cuda.current_stream())
    yield c
    c.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _problems():
    out = []
    p0 = scenes.config0()
    out.append(p0)
    p1 = scenes.config1(W=384, H=192)
    out.append(p1)
    p2 = scenes.trajectory_problem(250, 130, 3, seed_scene=1010)
    p2.params = dict(d_min=0.3, d_max=10.0, patch_w=9, patch_stride=3, iterations=3, best_k=2, sigma_color=0.15,
                     sigma_space=4.0, n_refine=6, neighbor_table=1, seed=5, keyframe_id=77)
    out.append(p2)
    p3 = scenes.trajectory_problem(320, 160, 8, seed_scene=1012, fmt="f16")
    p3.params = dict(p1.params, iterations=5, keyframe_id=9)
    out.append(p3)
    p4 = scenes.trajectory_problem(128, 64, 4, seed_scene=1013)
    p4.params = dict(p1.params, best_k=2, iterations=2, keyframe_id=11)
    out.append(p4)
    return out


def _args(p):
    return (_dev(p.ref.image), (p.ref.R, p.ref.t), [_dev(f.image) for f in p.srcs], [(f.R, f.t) for f in p.srcs])


def test_batch_equals_single_keyframe_runs(pm, ctx):
    """For view counts up to 10 the persistent batched kernel runs the paired
    per-pixel arithmetic of the single-keyframe kernels (view pairs in packed
    FP32, rotated column table), its constants read from shared memory instead
    of kernel parameters, so it matches single runs bit for bit; so do the
    per-keyframe chains, which run the single-keyframe kernels themselves."""
    probs = _problems()
    args = [_args(p) for p in probs]
    singles = [pm.pmsp_densify(ctx, *a, p.params).numpy() for a, p in zip(args, probs)]
    batch = pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)])
    outs = pm.pmsp_densify_batch(ctx, batch, tuning=pm.pmsp_tuning(0, 0, 0, 0))
    for (sd, sn, sc), o in zip(singles, outs):
        bd, bn, bc = o.numpy()
        assert np.array_equal(bc, sc) and np.array_equal(bd, sd) and np.array_equal(bn, sn)
    batch = pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)])
    outs = pm.pmsp_densify_batch(ctx, batch, tuning=pm.pmsp_tuning(0, 0, 0, 1))
    for (sd, sn, sc), o in zip(singles, outs):
        bd, bn, bc = o.numpy()
        assert np.array_equal(bc, sc) and np.array_equal(bd, sd) and np.array_equal(bn, sn)


def test_batch_with_more_than_ten_sources(pm, ctx):
    """A batch whose largest view count is above 10 runs the guarded 16-view
    instance of the persistent kernel (per-view arithmetic, views in shared
    memory): it matches the single-keyframe runs (exact 12- and 4-view kernels)
    within the parity tolerance; the per-keyframe chains run those kernels and
    match bit for bit."""
    pa = scenes.trajectory_problem(96, 48, 12, seed_scene=1014)
    pa.params = dict(d_min=0.3, d_max=10.0, patch_w=11, patch_stride=2, iterations=2, best_k=4, sigma_color=0.2,
                     sigma_space=3.0, n_refine=6, neighbor_table=0, seed=3, keyframe_id=21)
    pb = scenes.trajectory_problem(64, 32, 4, seed_scene=1015)
    pb.params = dict(pa.params, best_k=2, keyframe_id=22)
    probs = [pa, pb]
    args = [_args(p) for p in probs]
    singles = [pm.pmsp_densify(ctx, *a, p.params).numpy() for a, p in zip(args, probs)]
    for strategy in (0, 1):
        batch = pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)])
        outs = pm.pmsp_densify_batch(ctx, batch, tuning=pm.pmsp_tuning(0, 0, 0, strategy))
        for (sd, sn, sc), o in zip(singles, outs):
            bd, bn, bc = o.numpy()
            if strategy == 0:
                assert np.mean(np.abs(bc - sc) <= 1e-4) >= 0.995
                assert np.mean(np.abs(bd - sd) <= 5e-3 * sd) >= 0.995
            else:
                assert np.array_equal(bc, sc) and np.array_equal(bd, sd) and np.array_equal(bn, sn)


def test_tile_shapes_compute_the_same_numbers(pm, ctx):
    """Every tile shape of the fixed-window half-sweeps (32x8, 64x4, 16x16) runs
    the same per-pixel arithmetic, so the per-keyframe chains give bit-identical
    maps whatever the shape; problems with other windows ignore the shape."""
    probs = _problems()
    args = [_args(p) for p in probs]
    ref = None
    for tile in (0, 1, 2):
        batch = pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)])
        outs = [o.numpy() for o in pm.pmsp_densify_batch(ctx, batch, tuning=pm.pmsp_tuning(0, 0, 0, 1, tile))]
        if ref is None:
            ref = outs
            continue
        for (d0, n0, c0), (d1, n1, c1) in zip(ref, outs):
            assert np.array_equal(d0, d1) and np.array_equal(n0, n1) and np.array_equal(c0, c1)
    batch = pm.Batch([(*a, p.params, None) for a, p in zip(args[:1], probs[:1])])
    with pytest.raises(pm.PmspError) as e:
        pm.pmsp_densify_batch(ctx, batch, tuning=pm.pmsp_tuning(0, 0, 0, 1, 3))
    assert e.value.code == pm.PMSP_EINVAL


def test_batch_matches_oracle(pm, ctx):
    probs = _problems()[:3]
    args = [_args(p) for p in probs]
    outs = pm.pmsp_densify_batch(ctx, pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)]))
    for p, o in zip(probs, outs):
        od, on, oc = oracle.Problem.from_scene(p).densify()
        gd, _, gc = (x.astype(np.float64) for x in o.numpy())
        assert np.mean(np.abs(gd - od) / od <= 5e-3) >= 0.995
        assert np.mean(np.abs(gc - oc) <= 1e-4) >= 0.995


def test_graph_replay_and_host_batches(pm, ctx):
    probs = _problems()
    args = [_args(p) for p in probs]
    batch = pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)])
    first = [tuple(x.copy() for x in o.numpy()) for o in pm.pmsp_densify_batch(ctx, batch, pm.PMSP_BATCH_GRAPH)]
    for o in batch.outs:                       # poison the outputs, then replay the captured graph
        o.depth.fill_(-1.0)
    pm.pmsp_densify_batch(ctx, batch, pm.PMSP_BATCH_GRAPH)
    pm.pmsp_sync(ctx)
    for f, o in zip(first, batch.outs):
        for x, y in zip(f, o.numpy()):
            assert np.array_equal(x, y)
    # the same problems from host memory
    hb = pm.Batch([(p.ref.image, (p.ref.R, p.ref.t), [f.image for f in p.srcs], [(f.R, f.t) for f in p.srcs],
                    p.params, None) for p in probs])
    for f, o in zip(first, pm.pmsp_densify_batch(ctx, hb)):
        for x, y in zip(f, o.numpy()):
            assert np.array_equal(x, y)


def test_autotune_returns_valid_setting(pm, ctx):
    probs = _problems()[:2]
    args = [_args(p) for p in probs]
    batch = pm.Batch([(*a, dict(p.params, patch_stride=1, patch_w=7), None) for a, p in zip(args, probs)])
    t = pm.pmsp_autotune(ctx, batch, 0.01)
    assert t.strategy in (0, 1) and t.order in (0, 1) and t.patch_stride in (0, 2) and t.tile in (0, 1, 2)
    assert t.blocks_per_sm >= (1 if t.strategy == 0 else 0)
    outs = pm.pmsp_densify_batch(ctx, batch, 0, t)
    for o in outs:
        d = o.depth.cpu().numpy()
        assert np.all(np.isfinite(d)) and d.min() >= 0.3 - 1e-6 and d.max() <= 10.0 + 1e-5


def test_batch_rejects_bad_item(pm, ctx):
    probs = _problems()[:2]
    args = [_args(p) for p in probs]
    bad = dict(probs[1].params, best_k=9)
    with pytest.raises(pm.PmspError) as e:
        pm.pmsp_densify_batch(ctx, pm.Batch([(*args[0], probs[0].params, None), (*args[1], bad, None)]))
    assert e.value.code == pm.PMSP_EINVAL


@pytest.mark.parametrize("tpp", [1, 2, 4])
def test_threads_per_pixel_match_the_oracle(pm, ctx, tpp):
    """Half-sweeps with the views of each pixel split over tpp warps (the view
    pairs q = sub, sub + tpp, ... in warp `sub`, the odd last view in one of
    them, the views themselves above 10 sources), which exchange their view
    costs through shared memory: the maps equal the one-thread-per-pixel maps
    bit for bit (same sums in the same order, same sort), and the FP64 oracle's
    whole densification within the bar (cost 1e-4, range 0.5 % on 99.5 % of
    pixels). Problems: 6 views (3 pairs: uneven over 2 warps, one warp idle at
    4), 7 views in fp16 (an odd view), 12 views (6 pairs: 3 per warp at 2,
    uneven at 4), ragged tiles. The split kernels try every neighbour candidate
    in turn, while the one-thread kernel skips the bit-identical ones and pools
    the rest across the warp, so the equality also checks that pooling and
    skipping leave the maps unchanged."""
    p1 = scenes.config1(W=384, H=192)
    p2 = scenes.trajectory_problem(250, 130, 7, seed_scene=1016, fmt="f16")
    p2.params = dict(p1.params, iterations=3, best_k=2, keyframe_id=41)
    p3 = scenes.trajectory_problem(96, 48, 12, seed_scene=1014)
    p3.params = dict(d_min=0.3, d_max=10.0, patch_w=11, patch_stride=2, iterations=2, best_k=4, sigma_color=0.2,
                     sigma_space=3.0, n_refine=6, neighbor_table=0, seed=3, keyframe_id=21)
    probs = [p1, p2, p3]
    args = [_args(p) for p in probs]
    one = pm.pmsp_densify_batch(ctx, pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)]),
                                tuning=pm.pmsp_tuning(0, 0, 0, 1, 0, 1))
    one = [o.numpy() for o in one]
    outs = pm.pmsp_densify_batch(ctx, pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)]),
                                 tuning=pm.pmsp_tuning(0, 0, 0, 1, 0, tpp))
    for p, (wd, wn, wc), o in zip(probs, one, outs):
        gd, gn, gc = o.numpy()
        assert np.array_equal(gd, wd) and np.array_equal(gn, wn) and np.array_equal(gc, wc)
        od, on, oc = oracle.Problem.from_scene(p).densify()
        gd, gc = gd.astype(np.float64), gc.astype(np.float64)
        assert np.mean(np.abs(gd - od) / od <= 5e-3) >= 0.995
        assert np.mean(np.abs(gc - oc) <= 1e-4) >= 0.995


_LANE_ORACLE = {}


def _lane_problems():
    """Whole densifications for the lane split, with the FP64 oracle's maps (computed
    once for both lane counts)."""
    p1 = scenes.config1(W=384, H=192)
    p2 = scenes.trajectory_problem(250, 130, 7, seed_scene=1016, fmt="f16")
    p2.params = dict(p1.params, iterations=3, best_k=2, keyframe_id=41)
    p3 = scenes.trajectory_problem(96, 48, 12, seed_scene=1014)
    p3.params = dict(d_min=0.3, d_max=10.0, patch_w=11, patch_stride=2, iterations=2, best_k=4, sigma_color=0.2,
                     sigma_space=3.0, n_refine=6, neighbor_table=0, seed=3, keyframe_id=21)
    p4 = scenes.trajectory_problem(200, 100, 4, seed_scene=1017)
    p4.params = dict(p1.params, patch_w=5, patch_stride=1, iterations=3, best_k=2, keyframe_id=43)
    p5 = scenes.trajectory_problem(160, 80, 3, seed_scene=1018)
    p5.params = dict(p1.params, patch_w=3, patch_stride=1, iterations=3, best_k=1, sigma_color=0.0,
                     sigma_space=0.0, keyframe_id=44)
    probs = [p1, p2, p3, p4, p5]
    for k, p in enumerate(probs):
        if k not in _LANE_ORACLE:
            _LANE_ORACLE[k] = oracle.Problem.from_scene(p).densify()
    return probs, [_LANE_ORACLE[k] for k in range(len(probs))]


@pytest.mark.parametrize("tpp", [2, 4, 8])
def test_lane_split_matches_the_oracle(pm, ctx, tpp):
    """Half-sweeps with each pixel's patch samples split over tpp adjacent lanes of
    a warp (lane `sub` takes the samples sub, sub + tpp, ... of the window in
    row-major order, every lane the centre sample; 32x4, 32x2 or 32x1 tiles), whose four
    NCC sums per view
    and validity flag are combined by __shfl_xor_sync butterflies: the FP64
    oracle's whole densification within the bar (cost 1e-4, range 0.5 % on 99.5 %
    of pixels), and the one-thread maps within the same bar (the sums are added in
    another order, so not bit for bit). Problems: 6 views at 11x11 / 2 (35 samples
    besides the centre: 18 / 17 over 2 lanes, 9 / 8 over 4, 5 / 4 over 8), 7 views in fp16 (an
    odd view), 12 views (6 pairs), 4 views with a dense 5x5 window and 3 views with
    a 3x3 window and no bilateral weights (the generic window loop; at 3x3 a lane's
    samples wrap across rows), all with ragged tiles."""
    probs, ref = _lane_problems()
    args = [_args(p) for p in probs]
    one = pm.pmsp_densify_batch(ctx, pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)]),
                                tuning=pm.pmsp_tuning(0, 0, 0, 1, 0, 1))
    one = [o.numpy() for o in one]
    outs = pm.pmsp_densify_batch(ctx, pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)]),
                                 tuning=pm.pmsp_tuning(0, 0, 0, 1, 0, tpp, 1))
    for p, (wd, wn, wc), o, (od, on, oc) in zip(probs, one, outs, ref):
        gd, gn, gc = (a.astype(np.float64) for a in o.numpy())
        assert np.mean(np.abs(gd - od) / od <= 5e-3) >= 0.995
        assert np.mean(np.abs(gc - oc) <= 1e-4) >= 0.995
        assert np.mean(np.abs(gd - wd) / wd <= 5e-3) >= 0.995
        assert np.mean(np.abs(gc - wc) <= 1e-4) >= 0.995


def test_invalid_tuning_is_refused(pm, ctx):
    """Threads per pixel other than 0, 1, 2 or 4 (8 only with the lane split), a lane
    flag other than 0 or 1 and tile shapes outside 0..2 are refused with PMSP_EINVAL
    before anything runs; the context stays usable."""
    p = scenes.config0(W=64, H=32)
    args = _args(p)
    for bad in (pm.pmsp_tuning(0, 0, 0, 1, 0, 3), pm.pmsp_tuning(0, 0, 0, 1, 0, 8), pm.pmsp_tuning(0, 0, 0, 1, 3, 1),
                pm.pmsp_tuning(0, 0, 0, 1, 0, 2, 2), pm.pmsp_tuning(0, 0, 0, 1, 0, 2, -1),
                pm.pmsp_tuning(0, 0, 0, 1, 0, 16, 1)):
        with pytest.raises(pm.PmspError) as e:
            pm.pmsp_densify_batch(ctx, pm.Batch([(*args, p.params, None)]), tuning=bad)
        assert e.value.code == pm.PMSP_EINVAL
    pm.pmsp_densify_batch(ctx, pm.Batch([(*args, p.params, None)]), tuning=pm.pmsp_tuning(0, 0, 0, 1, 0, 2))
    pm.pmsp_densify_batch(ctx, pm.Batch([(*args, p.params, None)]), tuning=pm.pmsp_tuning(0, 0, 0, 1, 0, 4, 1))
    pm.pmsp_densify_batch(ctx, pm.Batch([(*args, p.params, None)]), tuning=pm.pmsp_tuning(0, 0, 0, 1, 0, 8, 1))
    pm.pmsp_sync(ctx)
