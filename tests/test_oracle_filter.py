"""Pins for the oracle's geometric-consistency filter.

Sec. III: once five depth maps exist the current one is checked against its
neighbours and outliers are removed, leaving an incomplete map. The project
reads this as a forward-backward reprojection test (error < 1 px in at least
2 neighbour views). Pins:

* exact ground-truth range maps are consistent almost everywhere away from
  the poles (near a pole one pixel of longitude is a tiny angle, so the
  nearest-pixel lookup's half-pixel error becomes many pixels there);
* corrupting one neighbour by +30 % range (a clear error at 256x128, where a
  pixel is 1.4 degrees) leaves the decision to the others;
* cameras sharing one centre cannot disagree on range: the decision is the
  same for any positive ranges, and under a yaw by whole pixels (the nearest
  pixel is the exact ray) every pixel agrees;
* a zero range (no data) in the neighbour never agrees; a zero reference
  range stays zero;
* rolling the reference map by k columns with its camera yawed by k pixels
  rolls every decision with it, also where the roll brings a pixel to the
  seam (the longitude error is wrapped to half a panorama).
"""
import numpy as np

import oracle
import scenes


def _frames(W=256, H=128, n=5):
    traj = scenes.trajectory(n, seed=2000)
    scene = scenes.Scene(seed=1001)
    scene.objects = scenes.place_objects(1078, [c for _, _, c in traj], n=20)
    out = []
    for (R, t, C) in traj:
        _, rg = scene.render(R, t, W, H, ss=1)
        out.append((R, t, rg))
    return out


def test_ground_truth_maps_are_consistent():
    fr = _frames()
    (Rr, tr, Dr) = fr[2]
    nb = [fr[i] for i in (0, 1, 3, 4)]
    out, agree, _ = oracle.consistency_filter(Dr, (Rr, tr), [d for _, _, d in nb],
                                              [(R, t) for R, t, _ in nb], 1.0, 2)
    band = slice(8, Dr.shape[0] - 8)
    assert np.mean(out[band] > 0) > 0.99
    assert np.mean(out[:3] > 0) < 0.5          # the pole rows mostly fail
    assert np.all((out == Dr) | (out == 0))
    assert np.mean(agree[band] == 4) > 0.75


def test_one_corrupted_view_is_outvoted():
    fr = _frames()
    (Rr, tr, Dr) = fr[2]
    nb = [fr[i] for i in (0, 1, 3, 4)]
    bad = [(R, t, d * (1.3 if i == 0 else 1.0)) for i, (R, t, d) in enumerate(nb)]
    out4, agree4, _ = oracle.consistency_filter(Dr, (Rr, tr), [d for _, _, d in bad],
                                                [(R, t) for R, t, _ in bad], 1.0, 2)
    band = slice(8, Dr.shape[0] - 8)
    assert np.mean(out4[band] > 0) > 0.95
    # with only the corrupted view and one good view, two agreeing views are rare
    two = [bad[0], bad[3]]
    out2, agree2, _ = oracle.consistency_filter(Dr, (Rr, tr), [d for _, _, d in two],
                                                [(R, t) for R, t, _ in two], 1.0, 2)
    good2 = [nb[0], nb[3]]
    outg, _, _ = oracle.consistency_filter(Dr, (Rr, tr), [d for _, _, d in good2],
                                           [(R, t) for R, t, _ in good2], 1.0, 2)
    assert np.mean(outg[band] > 0) > 0.75
    assert np.mean(out2[band] > 0) < 0.15


def test_shared_centre_agrees_for_any_range():
    rng = np.random.default_rng(0)
    W, H = 64, 32
    Dr = rng.uniform(0.5, 5.0, size=(H, W))
    C = [0.3, -0.2, 0.1]
    Rr, tr = scenes.pose_from_centre(scenes.rot_y(0.4), C)
    # yaw by a whole number of pixels: the nearest pixel is the exact ray, so
    # every view agrees whatever the neighbour's ranges are
    Rj, tj = scenes.pose_from_centre(scenes.rot_y(0.4 + 2 * np.pi * 5 / W), C)
    Dj = rng.uniform(0.5, 5.0, size=(H, W))
    out, agree, _ = oracle.consistency_filter(Dr, (Rr, tr), [Dj, 2 * Dj], [(Rj, tj), (Rj, tj)], 1.0, 2)
    assert np.array_equal(out, Dr)
    assert np.all(agree == 2)
    # any rotation about a shared centre: the decision does not depend on range
    Rk, tk = scenes.pose_from_centre(scenes.rot_y(1.1) @ scenes.rot_x(0.2), C)
    _, a1, _ = oracle.consistency_filter(Dr, (Rr, tr), [Dj], [(Rk, tk)], 1.0, 1)
    _, a2, _ = oracle.consistency_filter(Dr, (Rr, tr), [0.3 * Dj], [(Rk, tk)], 1.0, 1)
    _, a3, _ = oracle.consistency_filter(0.5 * Dr, (Rr, tr), [Dj], [(Rk, tk)], 1.0, 1)
    assert np.array_equal(a1, a2) and np.array_equal(a1, a3)
    assert a1[4:-4].mean() > 0.9
    # a neighbour without data never agrees
    out0, agree0, _ = oracle.consistency_filter(Dr, (Rr, tr), [Dj, np.zeros_like(Dj)],
                                                [(Rj, tj), (Rj, tj)], 1.0, 2)
    assert np.all(out0 == 0) and np.all(agree0 == 1)
    # a pixel without range stays without range
    Dz = Dr.copy()
    Dz[3, 5] = 0.0
    outz, agreez, _ = oracle.consistency_filter(Dz, (Rr, tr), [Dj, Dj], [(Rj, tj), (Rj, tj)], 1.0, 2)
    assert outz[3, 5] == 0 and agreez[3, 5] == 0


def test_min_views_threshold():
    fr = _frames(W=128, H=64)
    (Rr, tr, Dr) = fr[2]
    nb = [fr[i] for i in (0, 1, 3, 4)]
    Ds, Ps = [d for _, _, d in nb], [(R, t) for R, t, _ in nb]
    _, agree, _ = oracle.consistency_filter(Dr, (Rr, tr), Ds, Ps, 1.0, 1)
    for k in (1, 2, 3, 4):
        out, _, _ = oracle.consistency_filter(Dr, (Rr, tr), Ds, Ps, 1.0, k)
        assert np.array_equal(out > 0, agree >= k)


def test_decisions_follow_a_yaw_of_the_reference_across_the_seam():
    """Rolling the reference map by k columns while yawing its camera by k pixels
    (R' = Ry R, t' = Ry t with Ry turning longitude by 2 pi k / W) is the same
    physical map, so the agreeing-view counts roll with it, also for the pixels
    that the roll moves next to the seam. A neighbour at half the resolution
    makes round-trip errors of 0.5 to 1 px common, and those cross the seam at
    column 0 or W - 1 for some k."""
    W, H = 64, 32
    ref = _frames(W, H)[2]
    low = _frames(W // 2, H // 2)
    nb = [low[i] for i in (0, 1, 3, 4)]
    Rr, tr, Dr = ref
    kw = dict(nbr_depths=[d for _, _, d in nb], nbr_poses=[(R, t) for R, t, _ in nb], max_px=1.0, min_views=2)
    _, agree0, mg0 = oracle.consistency_filter(Dr, (Rr, tr), **kw)
    assert np.mean(agree0 > 0) > 0.5
    for k in range(1, W):
        a = 2 * np.pi * k / W
        Ry = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
        assert np.allclose(Ry @ oracle.bearing(W, H, 3, 7), oracle.bearing(W, H, 3 + k, 7), atol=1e-12)
        _, agree_k, mg_k = oracle.consistency_filter(np.roll(Dr, k, axis=1), (Ry @ Rr, Ry @ tr), **kw)
        clear = (np.roll(mg0, k, axis=1) > 1e-9) & (mg_k > 1e-9)
        assert np.array_equal(np.roll(agree0, k, axis=1)[clear], agree_k[clear]), k
