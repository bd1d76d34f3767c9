"""Pins for the oracle's PatchMatch: initialisation, propagation, refinement.

Sec. III-B (random initialisation) and Sec. III-C (red-black propagation over
an 8-neighbourhood, six shrinking random refinement tests) define the search;
the cost it minimises is pinned in test_oracle_cost.py. Here:

* the neighbour tables only reach the opposite colour;
* re-intersecting a neighbour's plane reproduces the exact range of a flat
  wall (closed form: a plane through the neighbour's wall point);
* a half-sweep equals independent per-pixel updates (order independence) and
  never raises a pixel's cost; the stored cost is the cost of the stored plane;
* the random initial planes and the refinement proposals come from Philox
  blocks laid out as (pixel, iteration, stage, 0) under key (seed, keyframe
  id), one uniform per perturbed component, checked with numpy's Philox;
* brute force: an exhaustive plane sweep (256 inverse-range levels x 162
  normals) on a tiny panorama does not beat the PatchMatch result by more than
  1e-3 on 95 % of pixels, and the final range is the sweep's optimum along the
  final normal within one level;
* on the rendered 256x128 room the result matches ground-truth range;
* the state never leaves the search space (ranges in [d_min, d_max], unit
  normals facing the camera) even when the true surface lies outside it.
"""

import numpy as np
import pytest

import oracle
import scenes


@pytest.mark.parametrize("table", [0, 1])
def test_neighbor_tables_reach_opposite_colour(table):
    nb = oracle.neighbor_table(table)
    assert len(nb) == 8 and len(set(nb)) == 8
    for dx, dy in nb:
        assert (dx + dy) % 2 == 1
        assert dx == 0 or dy == 0
    dist = sorted({abs(dx) + abs(dy) for dx, dy in nb})
    assert dist == ([3, 5] if table == 0 else [1, 5])


def _wall_state(prob):
    """Ground-truth range and camera-frame wall normals (room-only scene)."""
    gt = prob.ref.range
    H, W = gt.shape
    R, C = prob.ref.R, prob.ref.centre
    lo, hi = prob.scene.lo, prob.scene.hi
    n = np.zeros((3, H, W))
    wall = np.zeros((H, W), dtype=int)
    for v in range(H):
        for u in range(W):
            X = C + gt[v, u] * (R.T @ oracle.bearing(W, H, u, v))
            dl, dh = np.abs(X - lo), np.abs(X - hi)
            a = int(np.argmin(np.minimum(dl, dh)))
            side = 0 if dl[a] < dh[a] else 1
            nw = np.zeros(3)
            nw[a] = 1.0 if side == 0 else -1.0
            n[:, v, u] = R @ nw
            wall[v, u] = 2 * a + side
    return gt, n, wall


def test_propagation_recovers_flat_wall_range():
    prob = scenes.config0()
    pb = oracle.Problem.from_scene(prob, n_refine=0)
    gt, n, wall = _wall_state(prob)
    H, W = gt.shape
    depth, normal = gt.copy(), n.copy()
    cost = pb.cost_map(depth, normal)
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(400):
        u, v = int(rng.integers(0, W)), int(rng.integers(8, H - 8))
        rows = np.clip(np.arange(v - 8, v + 9), 0, H - 1)
        cols = np.arange(u - 8, u + 9) % W
        if np.any(wall[np.ix_(rows, cols)] != wall[v, u]):
            continue
        d0, n0, c0 = depth.copy(), normal.copy(), cost.copy()
        r = oracle.bearing(W, H, u, v)
        d0[v, u] = 0.6 * gt[v, u]
        n0[:, v, u] = -r
        c0[v, u] = pb.cost(u, v, d0[v, u], -r)
        d, nn, c = pb.update_pixel(d0, n0, c0, u, v, 0)
        assert abs(d - gt[v, u]) < 1e-9 * gt[v, u]
        np.testing.assert_allclose(nn, n[:, v, u], atol=1e-12)
        assert c < c0[v, u]
        checked += 1
        if checked >= 12:
            break
    assert checked >= 6


def test_halfsweep_is_order_independent_and_monotone():
    prob = scenes.config0()
    pb = oracle.Problem.from_scene(prob)
    d, n, c = pb.init()
    for it in range(2):
        for colour in (0, 1):
            d0, n0, c0 = d.copy(), n.copy(), c.copy()
            pb.halfsweep(d, n, c, colour, it)
            assert np.all(c <= c0)
            H, W = d.shape
            vv, uu = np.nonzero(((np.arange(W)[None, :] + np.arange(H)[:, None]) % 2) != colour)
            assert np.array_equal(d[vv, uu], d0[vv, uu])       # other colour untouched
            rng = np.random.default_rng(it * 2 + colour)
            for _ in range(40):
                v = int(rng.integers(0, H))
                u = int(rng.integers(0, W // 2)) * 2 + ((v + colour) & 1)
                du, nu, cu = pb.update_pixel(d0, n0, c0, u, v, it)
                assert du == d[v, u] and cu == c[v, u]
                assert np.array_equal(nu, n[:, v, u])
    # stored cost is the cost of the stored plane
    np.testing.assert_allclose(pb.cost_map(d, n), c, atol=1e-12, rtol=0)


def test_random_init_draw_layout():
    prob = scenes.config0()
    pb = oracle.Problem.from_scene(prob, seed=7, keyframe_id=9)
    H, W = prob.ref.image.shape
    dmin, dmax = 0.3, 10.0
    for (u, v) in [(0, 0), (5, 3), (W - 1, H - 1), (100, 64)]:
        d, n = pb.random_plane(u, v)
        p = v * W + u
        bg = np.random.Philox(key=np.array([7, 9], dtype=np.uint64),
                              counter=np.array([p - 1 if p else 2**64 - 1, 0 if p else 2**64 - 1,
                                                0 if p else 2**64 - 1, 0 if p else 2**64 - 1],
                                               dtype=np.uint64))
        w = bg.random_raw(4)
        u0 = int(w[0]) >> 40
        inv = 1 / dmax + (u0 / 2**24) * (1 / dmin - 1 / dmax)
        assert abs(d - 1 / inv) < 1e-12 * d
        r = oracle.bearing(W, H, u, v)
        assert n @ r < 0 and abs(np.linalg.norm(n) - 1) < 1e-12
        z = 1 - 2 * ((int(w[1]) >> 40) / 2**24)
        assert abs(abs(n[2]) - abs(z)) < 1e-12 or np.allclose(n, -r)


def test_random_init_distribution():
    prob = scenes.config0()
    pb = oracle.Problem.from_scene(prob)
    d, n, _ = pb.init()
    inv = 1.0 / d
    lo, hi = 1 / 10.0, 1 / 0.3
    assert inv.min() >= lo - 1e-12 and inv.max() <= hi
    # uniform in inverse range: mean and quartiles
    x = (inv - lo) / (hi - lo)
    assert abs(x.mean() - 0.5) < 0.01
    assert abs(np.quantile(x, 0.25) - 0.25) < 0.01
    H, W = d.shape
    r = np.stack([oracle.bearing(W, H, u, v) for v in range(H) for u in range(W)], 1).reshape(3, H, W)
    assert np.all(np.sum(n * r, axis=0) < 0)


def _icosphere(level):
    t = (1 + 5 ** 0.5) / 2
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
         (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]
        NF = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            NF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = NF
    return np.array(V)


def test_config0_matches_ground_truth():
    prob = scenes.config0()
    pb = oracle.Problem.from_scene(prob)
    d, n, c = pb.densify()
    rel = np.abs(d - prob.ref.range) / prob.ref.range
    assert np.mean(rel < 0.05) > 0.9
    assert np.mean(rel < 0.01) > 0.5
    assert np.median(c) < 0.02


def test_state_stays_in_the_search_space():
    """The search space of Sec. III-B/C is ranges in [d_min, d_max] and unit normals
    facing the camera; propagation re-intersections and refinement proposals that
    leave it are not taken. A range window narrower than the room (part of the true
    surface lies beyond d_max) makes out-of-window candidates the better fit, so a
    missing bound would show."""
    W, H = 48, 24
    scene = scenes.Scene(seed=1234)
    C = np.array([0.2, 0.1, -0.3])
    R0, t0 = scenes.pose_from_centre(scenes.rot_y(0.3), C)
    views = [scenes.pose_from_centre(scenes.rot_y(0.3), C + np.array(o)) for o in ((0.2, 0, 0), (0, 0, 0.2))]
    img0, rng0 = scene.render(R0, t0, W, H)
    imgs = [scene.render(R, t, W, H)[0] / 255.0 for R, t in views]
    d_min, d_max = 0.5, 2.0
    assert np.mean(rng0 > d_max) > 0.2
    pb = oracle.Problem(img0 / 255.0, (R0, t0), imgs, views, d_min=d_min, d_max=d_max, patch_w=7,
                        patch_stride=1, iterations=6, best_k=1)
    d, n, c = pb.densify()
    assert np.all((d >= d_min * (1 - 1e-12)) & (d <= d_max * (1 + 1e-12)))
    assert np.allclose(np.sum(n * n, 0), 1.0, atol=1e-12)
    r = np.stack([oracle.bearing(W, H, u, v) for v in range(H) for u in range(W)]).reshape(H, W, 3)
    assert np.all(np.sum(n * r.transpose(2, 0, 1), 0) < 0)
    assert np.array_equal(c, pb.cost_map(d, n))


def _philox_block(seed, keyframe_id, counter):
    """The Philox4x64-10 block at a 256-bit counter, from numpy's generator (which
    advances its counter before each block, so it is started one below)."""
    c = (sum(int(w) << (64 * i) for i, w in enumerate(counter)) - 1) % (1 << 256)
    ctr = np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    return np.random.Philox(key=np.array([seed, keyframe_id], dtype=np.uint64), counter=ctr).random_raw(4)


def test_refinement_draw_layout():
    """With the incumbent's cost above any cost (5 > 2) and every neighbour plane facing
    away (never re-intersected), the first refinement test of a half-sweep is always
    taken, so one test exposes its proposal: the range and normal perturbations of
    Sec. III-C built from the Philox block at counter (pixel, iteration, 1, 0) under key
    (seed, keyframe id), checked with numpy's Philox, one uniform per component."""
    W, H, seed, kf, it, colour = 64, 32, 13, 4, 2, 1
    scene = scenes.Scene(seed=1234)
    C = np.array([0.2, 0.1, -0.3])
    R0, t0 = scenes.pose_from_centre(scenes.rot_y(0.3), C)
    R1, t1 = scenes.pose_from_centre(scenes.rot_y(0.3), C + np.array([0.2, 0.0, 0.0]))
    img0, _ = scene.render(R0, t0, W, H)
    img1, _ = scene.render(R1, t1, W, H)
    d_min, d_max = 0.3, 10.0
    pb = oracle.Problem(img0 / 255.0, (R0, t0), [img1 / 255.0], [(R1, t1)], d_min=d_min, d_max=d_max, patch_w=5,
                        patch_stride=1, iterations=1, best_k=1, n_refine=1, seed=seed, keyframe_id=kf)
    r = np.stack([oracle.bearing(W, H, u, v) for v in range(H) for u in range(W)], 1).reshape(3, H, W)
    rng = np.random.default_rng(1)
    d0 = rng.uniform(0.5, 5.0, (H, W))
    n0 = -r + 0.3 * rng.normal(size=(3, H, W))
    n0 /= np.linalg.norm(n0, axis=0)
    n0 = np.where(np.sum(n0 * r, 0) < 0, n0, -n0)
    other = ((np.arange(W)[None, :] + np.arange(H)[:, None]) % 2) != colour
    n0[:, other] = r[:, other]
    d, n, c = d0.copy(), np.ascontiguousarray(n0).copy(), np.full((H, W), 5.0)
    pb.halfsweep(d, n, c, colour, it)
    for (u, v) in [(1, 0), (0, 1), (W - 1, 0), (17, 8), (40, 15), (33, 30), (W - 2, H - 1)]:
        assert (u + v) % 2 == colour
        p = v * W + u
        uu = [(int(x) >> 40) / 2**24 for x in _philox_block(seed, kf, [p, it, 1, 0])]
        s = 0.5
        inv = 1 / d0[v, u] + (2 * uu[0] - 1) * s * (1 / d_min - 1 / d_max)
        inv = min(max(inv, 1 / d_max), 1 / d_min)
        assert abs(d[v, u] - 1 / inv) <= 1e-12 * d[v, u]
        m = n0[:, v, u] + s * (2 * np.array(uu[1:]) - 1)
        m /= np.linalg.norm(m)
        cr = m @ r[:, v, u]
        m = -r[:, v, u] if abs(cr) < 1e-3 else (-m if cr > 0 else m)
        assert np.allclose(n[:, v, u], m, atol=1e-12, rtol=0)
        assert c[v, u] <= 2.0
    assert np.array_equal(d[other], d0[other])


def test_refinement_schedule_shrinks_around_current_best():
    """The six refinement tests of Sec. III-C, seen one at a time through
    n_refine = 1..6 from the same state (incumbent cost above any cost, every
    neighbour facing away): result m equals result m - 1 or has a strictly lower
    cost; an accepted test m moves the inverse range at most s_m (1/d_min -
    1/d_max) from result m - 1 (the current best, not the half-sweep's starting
    plane), s_m = 2^-m, and over many pixels the moves fill that bound (each
    test draws its own uniform), so the search range halves at every test."""
    W, H, seed, kf, it, colour = 64, 32, 21, 6, 3, 0
    scene = scenes.Scene(seed=1234)
    C = np.array([0.2, 0.1, -0.3])
    R0, t0 = scenes.pose_from_centre(scenes.rot_y(0.3), C)
    R1, t1 = scenes.pose_from_centre(scenes.rot_y(0.3), C + np.array([0.2, 0.0, 0.0]))
    img0, _ = scene.render(R0, t0, W, H)
    img1, _ = scene.render(R1, t1, W, H)
    d_min, d_max = 0.3, 10.0
    span = 1 / d_min - 1 / d_max
    r = np.stack([oracle.bearing(W, H, u, v) for v in range(H) for u in range(W)], 1).reshape(3, H, W)
    rng = np.random.default_rng(2)
    d0 = rng.uniform(0.5, 5.0, (H, W))
    n0 = -r + 0.3 * rng.normal(size=(3, H, W))
    n0 /= np.linalg.norm(n0, axis=0)
    n0 = np.where(np.sum(n0 * r, 0) < 0, n0, -n0)
    act = ((np.arange(W)[None, :] + np.arange(H)[:, None]) % 2) == colour
    n0[:, ~act] = r[:, ~act]
    chain = [(d0, np.full((H, W), 5.0))]
    for m in range(1, 7):
        pb = oracle.Problem(img0 / 255.0, (R0, t0), [img1 / 255.0], [(R1, t1)], d_min=d_min, d_max=d_max,
                            patch_w=5, patch_stride=1, iterations=1, best_k=1, n_refine=m, seed=seed,
                            keyframe_id=kf)
        d, n, c = d0.copy(), np.ascontiguousarray(n0).copy(), np.full((H, W), 5.0)
        pb.halfsweep(d, n, c, colour, it)
        chain.append((d, c))
    for m in range(1, 7):
        (dp, cp), (dm, cm) = chain[m - 1], chain[m]
        moved = act & (dm != dp)
        assert np.all(cm[act] <= cp[act])
        assert np.all(cm[moved] < cp[moved])
        step = np.abs(1 / dm - 1 / dp)[moved] / (2.0 ** -m * span)
        assert np.all(step <= 1 + 1e-9), (m, step.max())
        assert moved.sum() >= 40, (m, moved.sum())
        assert step.max() >= 0.8, (m, step.max())


def test_patchmatch_reaches_exhaustive_sweep_minimum():
    """Brute force on a tiny input: a 32x16 panorama, one source 0.2 m to the
    side, 7x7 window. (1) An exhaustive sweep over 256 inverse-range levels x
    162 icosphere normals (level 2) does not beat the PatchMatch cost after
    128 iterations by more than 1e-3 on 95 % of pixels. (2) The final plane
    is a depth optimum along its own normal: a sweep of the same 256 levels
    with that normal finds its minimum within one level of the PatchMatch
    range on 98 % of pixels and no cost below it by more than 1e-3 on 99 %.
    Part (2) states the depth check on the PatchMatch plane's own normal
    because the continuous normals beat the 162 sampled ones on almost every
    pixel, so the 2-D sweep's argmin range carries the normal sampling's bias.
    (Measured on the oracle: 97.3 %, 99.2 %, 100 %; with 16 iterations 67 %
    and 80 %: the pin needs a search that converges.)"""
    W, H = 32, 16
    scene = scenes.Scene(seed=1234)
    C = np.array([0.2, 0.1, -0.3])
    R0, t0 = scenes.pose_from_centre(scenes.rot_y(0.3), C)
    R1, t1 = scenes.pose_from_centre(scenes.rot_y(0.3), C + np.array([0.2, 0.0, 0.0]))
    img0, _ = scene.render(R0, t0, W, H)
    img1, _ = scene.render(R1, t1, W, H)
    pb = oracle.Problem(img0 / 255.0, (R0, t0), [img1 / 255.0], [(R1, t1)], patch_w=7,
                        patch_stride=1, iterations=128, best_k=1)
    N = _icosphere(2)
    assert len(N) == 162
    L = 256
    sweep_cost, _ = pb.plane_sweep(L, N)
    d, n, c = pb.densify()
    assert np.mean(c <= sweep_cost + 1e-3) >= 0.95
    inv = 1.0 / 10.0 + (1.0 / 0.3 - 1.0 / 10.0) * np.arange(L) / (L - 1)
    level = np.zeros((H, W))
    gap = np.zeros((H, W))
    for v in range(H):
        for u in range(W):
            line = np.array([pb.cost(u, v, 1.0 / x, n[:, v, u]) for x in inv])
            k = int(np.argmin(line))
            level[v, u] = abs(1.0 / d[v, u] - inv[k]) / (inv[1] - inv[0])
            gap[v, u] = c[v, u] - line[k]
    assert np.mean(level <= 1.0) >= 0.98
    assert np.mean(gap <= 1e-3) >= 0.99
