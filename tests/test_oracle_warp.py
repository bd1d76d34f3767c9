"""Pins for the oracle's plane-map warping initialisation (Sec. III-B).

The preceding keyframe's plane map is moved into the current keyframe: each
plane is splatted to the nearest current pixel (nearest surface wins) and
re-intersected with that pixel's ray; pixels no plane reaches start from the
random initialisation. Pins:

* the same camera: every plane lands on its own pixel unchanged;
* a yaw by exactly k pixels about the camera centre: planes land k columns
  over with their ranges unchanged and their normals rotated;
* a translated camera looking at the flat walls of the room: the warped range
  is the wall's range along the new ray (closed form), wherever the whole
  neighbourhood sees the same wall;
* the winner of every pixel is the nearest of the planes that land on it
  (brute force over all previous pixels);
* pixels without a plane hold exactly the random initial plane.
"""
import math

import numpy as np

import oracle
import scenes


def _room_frames(W=128, H=64, n=4, seed=2000):
    traj = scenes.trajectory(n, seed=seed)
    scene = scenes.Scene(seed=1001)
    out = []
    for (R, t, C) in traj:
        img, rg = scene.render(R, t, W, H)
        out.append(dict(img=scenes.quantise_u8(img), R=R, t=t, C=C, range=rg))
    return scene, out


def _wall_planes(scene, f):
    """Ground-truth range and camera-frame wall normal of every pixel (room only)."""
    H, W = f["range"].shape
    n = np.zeros((3, H, W))
    wall = np.zeros((H, W), int)
    for v in range(H):
        for u in range(W):
            X = f["C"] + f["range"][v, u] * (f["R"].T @ oracle.bearing(W, H, u, v))
            dl, dh = np.abs(X - scene.lo), np.abs(X - scene.hi)
            a = int(np.argmin(np.minimum(dl, dh)))
            side = 0 if dl[a] < dh[a] else 1
            nw = np.zeros(3)
            nw[a] = 1.0 if side == 0 else -1.0
            n[:, v, u] = f["R"] @ nw
            wall[v, u] = 2 * a + side
    return f["range"].copy(), n, wall


def _problem(f, srcs):
    return oracle.Problem(f["img"], (f["R"], f["t"]), [s["img"] for s in srcs], [(s["R"], s["t"]) for s in srcs],
                          patch_w=5, patch_stride=1, best_k=1)


def test_same_camera_keeps_every_plane():
    scene, fr = _room_frames()
    d0, n0, _ = _wall_planes(scene, fr[1])
    pb = _problem(fr[1], [fr[0]])
    d, n, c, src, clear = pb.warp_init(d0, n0, (fr[1]["R"], fr[1]["t"]), (fr[1]["R"], fr[1]["t"]))
    H, W = d0.shape
    assert np.array_equal(src.ravel(), np.arange(W * H))
    np.testing.assert_allclose(d, d0, rtol=1e-9)
    np.testing.assert_allclose(n, n0, atol=1e-12)
    np.testing.assert_allclose(c, pb.cost_map(d, n), atol=1e-12)


def test_yaw_by_whole_pixels_moves_planes_k_columns():
    scene, fr = _room_frames()
    H, W = fr[1]["range"].shape
    d0, n0, _ = _wall_planes(scene, fr[1])
    k = 5
    yaw = 2 * math.pi * k / W
    Rc = scenes.rot_y(yaw) @ fr[1]["R"]          # world->camera of a camera turned by k pixels
    tc = -Rc @ fr[1]["C"]
    cur = dict(fr[1], R=Rc, t=tc)
    pb = _problem(cur, [fr[0]])
    d, n, c, src, clear = pb.warp_init(d0, n0, (fr[1]["R"], fr[1]["t"]), (Rc, tc))
    Rrel = scenes.rot_y(yaw)
    for v in range(1, H - 1):
        for u in range(W):
            j = src[v, u]
            assert j == v * W + (u - k) % W
            assert abs(d[v, u] - d0.ravel()[j]) < 1e-9 * d[v, u]
            np.testing.assert_allclose(n[:, v, u], Rrel @ n0[:, j // W, j % W], atol=1e-12)


def test_translation_reproduces_wall_range():
    scene, fr = _room_frames()
    d0, n0, wall0 = _wall_planes(scene, fr[1])
    _, _, wall2 = _wall_planes(scene, fr[2])
    pb = _problem(fr[2], [fr[1]])
    d, n, c, src, clear = pb.warp_init(d0, n0, (fr[1]["R"], fr[1]["t"]), (fr[2]["R"], fr[2]["t"]))
    gt = fr[2]["range"]
    H, W = gt.shape
    checked = 0
    for v in range(4, H - 4):
        for u in range(W):
            j = src[v, u]
            if j < 0:
                continue
            cols = np.arange(u - 3, u + 4) % W
            if np.any(wall2[v - 3:v + 4][:, cols] != wall2[v, u]) or wall0.ravel()[j] != wall2[v, u]:
                continue
            assert abs(d[v, u] - gt[v, u]) < 1e-9 * gt[v, u]
            checked += 1
    assert checked > W * H // 3


def test_nearest_plane_wins_and_holes_are_random():
    W, H = 96, 48
    traj = scenes.trajectory(3, seed=2001)
    scene = scenes.Scene(seed=1005)
    scene.objects = scenes.place_objects(1082, [c for _, _, c in traj], n=20)
    fr = []
    for (R, t, C) in traj:
        img, rg = scene.render(R, t, W, H)
        fr.append(dict(img=scenes.quantise_u8(img), R=R, t=t, C=C, range=rg))
    rng = np.random.default_rng(0)
    d0 = fr[0]["range"].copy()
    d0[rng.uniform(size=d0.shape) < 0.2] = 0.0                    # holes in the previous map
    n0 = -np.stack([oracle.bearing(W, H, u, v) for v in range(H) for u in range(W)], 1).reshape(3, H, W)
    pb = _problem(fr[1], [fr[2]])
    d, n, c, src, clear = pb.warp_init(d0, n0, (fr[0]["R"], fr[0]["t"]), (fr[1]["R"], fr[1]["t"]))
    Rrel, trel = oracle.rel_pose(fr[0]["R"], fr[0]["t"], fr[1]["R"], fr[1]["t"])
    land = {}
    for v in range(H):
        for u in range(W):
            if d0[v, u] <= 0:
                continue
            Y = Rrel @ (d0[v, u] * oracle.bearing(W, H, u, v)) + trel
            uc, vc = oracle.project(W, H, Y)
            q = (min(max(int(math.floor(vc + 0.5)), 0), H - 1), int(math.floor(uc + 0.5)) % W)
            land.setdefault(q, []).append((np.linalg.norm(Y), v * W + u))
    for (qv, qu), cands in land.items():
        if src[qv, qu] >= 0:
            assert src[qv, qu] == min(cands)[1]
    holes = 0
    for v in range(H):
        for u in range(W):
            if src[v, u] < 0:
                dr, nr = pb.random_plane(u, v)
                assert d[v, u] == dr and np.array_equal(n[:, v, u], nr)
                holes += 1
    assert 0 < holes < W * H
