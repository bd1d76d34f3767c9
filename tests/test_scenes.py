"""Pins for the synthetic scene generator (inputs shared by oracle and CUDA path).

Closed forms: the range from a camera inside the empty room to the wall it
faces is the distance to that wall plane divided by the direction cosine; a
sphere seen head-on is at centre distance minus radius. Determinism by seed.
"""
import math

import numpy as np

import scenes


def test_room_range_closed_form():
    s = scenes.Scene(seed=5)
    o = np.array([0.3, -0.2, 0.4])
    dirs = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]], float)
    rg = s.ray_range(np.repeat(o[None], 6, 0), dirs)
    expect = [1.5 - 0.4, 0.4 + 1.5, 2.0 - 0.3, 0.3 + 2.0, 1.25 + 0.2, 1.25 - 0.2]
    np.testing.assert_allclose(rg, expect, atol=1e-12)
    d = np.array([0.3, 0.1, 1.0])
    d /= np.linalg.norm(d)
    r = s.ray_range(o[None], d[None])[0]
    assert abs(r - (1.5 - 0.4) / d[2]) < 1e-12


def test_rendered_range_matches_wall_planes():
    s = scenes.Scene(seed=6)
    C = np.array([0.1, 0.2, -0.3])
    R, t = scenes.pose_from_centre(np.eye(3), C)
    W, H = 64, 32
    _, rg = s.render(R, t, W, H, ss=1)
    for v in range(4, H - 4):
        for u in range(W):
            lon = 2 * math.pi * (u + 0.5) / W - math.pi
            lat = math.pi / 2 - math.pi * (v + 0.5) / H
            b = np.array([math.cos(lat) * math.sin(lon), -math.sin(lat), math.cos(lat) * math.cos(lon)])
            ts = [((scenes.ROOM_HI[a] if b[a] > 0 else scenes.ROOM_LO[a]) - C[a]) / b[a]
                  for a in range(3) if abs(b[a]) > 1e-12]
            assert abs(rg[v, u] - min(ts)) < 1e-9


def test_sphere_head_on():
    s = scenes.Scene(seed=7)
    s.objects = [scenes.SceneObject(0, np.array([0.0, 0.0, 1.0]), 0.3, 3, 0.5, 0.2)]
    rg = s.ray_range(np.zeros((1, 3)), np.array([[0, 0, 1.0]]))
    assert abs(rg[0] - 0.7) < 1e-12


def test_deterministic_by_seed_and_texture_present():
    a = scenes.config0()
    b = scenes.config0()
    assert np.array_equal(a.ref.image, b.ref.image)
    assert np.array_equal(a.srcs[1].image, b.srcs[1].image)
    assert a.ref.image.std() > 10
    c = scenes.config0(seed=1001)
    assert not np.array_equal(a.ref.image, c.ref.image)


def test_trajectory_statistics():
    traj = scenes.trajectory(200, seed=2000)
    C = np.array([c for _, _, c in traj])
    steps = np.linalg.norm(np.diff(C, axis=0), axis=1)
    assert 0.1 < steps.mean() < 0.2
    assert np.all(C >= scenes.ROOM_LO + 0.4 - 1e-9) and np.all(C <= scenes.ROOM_HI - 0.4 + 1e-9)
    for (R0, _, _), (R1, _, _) in zip(traj[:-1], traj[1:]):
        ang = math.degrees(math.acos(np.clip((np.trace(R0 @ R1.T) - 1) / 2, -1, 1)))
        assert ang < 10 + 2 * 5 * 1.5     # yaw <= 10 deg plus bounded pitch/roll jitter
    objs = scenes.place_objects(1078, C, n=20)
    for o in objs:
        assert 0.2 <= o.radius <= 1.0
        d = scenes._obj_distance(o.kind, o.centre, o.radius, C)
        assert np.all(d > 0.3)
