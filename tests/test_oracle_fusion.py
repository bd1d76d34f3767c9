"""Pins for the oracle's point-cloud fusion (Sec. III) and completeness (Sec. IV).

Fusion: the back-projected ground-truth range of a room-only render lies on
the room's walls (closed form), a keyframe fused with itself adds nothing,
the kept point of each voxel is the first in (keyframe, pixel) order (brute
force over points computed from the camera centres and closed-form bearings
on a tiny input), and reordering keyframes keeps the voxel set.
Completeness: one point per pixel ray covers the panorama exactly, a single
point covers one pixel, and a keyframe's own cloud seen from its own pose at
its own resolution hits exactly its valid pixels.
"""
import numpy as np

import oracle
import scenes


def _bearing(W, H):
    u, v = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    lon = 2 * np.pi * u / W - np.pi
    lat = np.pi / 2 - np.pi * v / H
    return np.stack([np.cos(lat) * np.sin(lon), -np.sin(lat), np.cos(lat) * np.cos(lon)], -1)


def _room_view(W=64, H=32, C=(0.3, -0.2, 0.1), yaw=0.5):
    scene = scenes.Scene(seed=7)
    scene.objects = []
    R, t = scenes.pose_from_centre(scenes.rot_y(yaw) @ scenes.rot_x(0.1), np.array(C))
    _, rng = scene.render(R, t, W, H, ss=1)
    return (R, t), rng


def test_room_points_lie_on_walls():
    pose, rng = _room_view()
    pts, src, _ = oracle.fuse([rng], [pose], voxel=1e-4)
    lo, hi = scenes.ROOM_LO, scenes.ROOM_HI
    dist = np.min(np.concatenate([np.abs(pts - lo), np.abs(pts - hi)], 1), 1)
    assert np.max(dist) < 1e-9
    assert np.all((pts >= lo - 1e-9) & (pts <= hi + 1e-9))


def test_self_fusion_adds_nothing_and_keeps_first_keyframe():
    pose, rng = _room_view()
    p1, s1, _ = oracle.fuse([rng], [pose], voxel=0.05)
    p2, s2, _ = oracle.fuse([rng, rng], [pose, pose], voxel=0.05)
    assert np.array_equal(p1, p2) and np.array_equal(s1, s2)
    assert np.all((s2 >> 32) == 0)


def test_first_point_per_voxel_brute_force():
    W, H, voxel = 16, 8, 0.237  # walls (multiples of 0.25 m) stay off voxel faces
    views = [_room_view(W, H, C=c, yaw=y) for c, y in (((0.3, -0.2, 0.1), 0.5), ((0.1, 0.0, -0.2), 2.0))]
    views[1][1][2, 3] = 0.0                      # a hole: no point
    pts, src, _ = oracle.fuse([r for _, r in views], [p for p, _ in views], voxel=voxel)
    first = {}
    b = _bearing(W, H).reshape(-1, 3)
    for k, ((R, t), rng) in enumerate(views):
        C = -R.T @ t
        for i, d in enumerate(rng.reshape(-1)):
            if d <= 0:
                continue
            X = C + R.T @ (d * b[i])
            key = tuple(np.floor(X / voxel).astype(np.int64))
            first.setdefault(key, (k << 32) | i)
    assert len(src) == len(first)
    keys = [tuple(np.floor(p / voxel).astype(np.int64)) for p in pts]
    assert keys == sorted(keys)
    assert [first[k] for k in keys] == src.tolist()


def test_keyframe_order_keeps_voxel_set():
    a, b = _room_view(C=(0.3, -0.2, 0.1), yaw=0.5), _room_view(C=(-0.4, 0.1, 0.2), yaw=-1.0)
    p1, _, _ = oracle.fuse([a[1], b[1]], [a[0], b[0]], voxel=0.097)
    p2, _, _ = oracle.fuse([b[1], a[1]], [b[0], a[0]], voxel=0.097)
    k1 = np.floor(p1 / 0.097).astype(np.int64)
    k2 = np.floor(p2 / 0.097).astype(np.int64)
    assert np.array_equal(k1, k2)


def test_completeness_one_point_per_pixel_ray():
    W, H = 72, 36
    R, t = scenes.pose_from_centre(scenes.rot_y(0.3), np.array([0.2, 0.1, -0.3]))
    C = -R.T @ t
    pts = C + 2.0 * (_bearing(W, H).reshape(-1, 3) @ R)
    c, hit, margin = oracle.completeness(pts, (R, t), W, H)
    assert c == 1.0 and hit.all()
    assert np.min(margin) > 0.49
    c1, hit1, _ = oracle.completeness(pts[:1], (R, t), W, H)
    assert c1 == 1.0 / (W * H) and hit1.sum() == 1 and hit1[0, 0]
    c0, _, _ = oracle.completeness(np.zeros((0, 3)), (R, t), W, H)
    assert c0 == 0.0


def test_completeness_of_own_cloud_equals_valid_share():
    pose, rng = _room_view(48, 24)
    rng = rng.copy()
    rng[np.random.default_rng(0).random(rng.shape) < 0.3] = 0.0
    pts, _, _ = oracle.fuse([rng], [pose], voxel=1e-5)
    c, hit, _ = oracle.completeness(pts, pose, 48, 24)
    assert np.array_equal(hit, rng > 0)
    assert c == np.mean(rng > 0)
