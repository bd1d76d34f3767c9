"""Pins for the oracle's equirectangular camera, pose composition and sampling.

The paper only names the camera ("equirectangular", Sec. III-C); the project
fixes the convention (x right, y down, z forward; pixel centres at
lon = 2*pi*(u+0.5)/W - pi, lat = pi/2 - pi*(v+0.5)/H). These tests pin the
oracle to closed-form bearings, the projection round trip, the seam, pose
composition as an identity on points, and bilinear reproduction of linear
images.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("W,H", [(8, 4), (256, 128), (1920, 960)])
def test_cardinal_bearings(W, H):
    c = lambda u, v: oracle.bearing(W, H, u, v)
    np.testing.assert_allclose(c(W / 2 - 0.5, H / 2 - 0.5), [0, 0, 1], atol=1e-12)     # forward
    np.testing.assert_allclose(c(3 * W / 4 - 0.5, H / 2 - 0.5), [1, 0, 0], atol=1e-12)  # right
    np.testing.assert_allclose(c(W / 4 - 0.5, H / 2 - 0.5), [-1, 0, 0], atol=1e-12)     # left
    np.testing.assert_allclose(c(-0.5, H / 2 - 0.5), [0, 0, -1], atol=1e-12)            # back
    np.testing.assert_allclose(c(W / 2 - 0.5, -0.5), [0, -1, 0], atol=1e-12)            # zenith (y down)
    np.testing.assert_allclose(c(W / 2 - 0.5, H - 0.5), [0, 1, 0], atol=1e-12)          # nadir


def test_bearing_unit_and_latitude_rows():
    W, H = 64, 32
    for v in range(H):
        lat = math.pi / 2 - math.pi * (v + 0.5) / H
        for u in (0, 17, 63):
            r = oracle.bearing(W, H, u, v)
            assert abs(np.linalg.norm(r) - 1) < 1e-14
            assert abs(-r[1] - math.sin(lat)) < 1e-14


def test_project_round_trip_and_scale_invariance():
    W, H = 1920, 960
    rng = np.random.default_rng(0)
    for _ in range(500):
        u = rng.uniform(-0.5, W - 0.5)
        v = rng.uniform(1.0, H - 2.0)            # away from the two pole rows
        r = oracle.bearing(W, H, u, v)
        uc, vc = oracle.project(W, H, r)
        du = (uc - u + W / 2) % W - W / 2
        assert abs(du) < 1e-8 and abs(vc - v) < 1e-8
        uc2, vc2 = oracle.project(W, H, 3.7 * r)
        assert abs(uc2 - uc) < 1e-9 and abs(vc2 - vc) < 1e-9


def test_seam_columns_are_neighbours():
    W, H = 256, 128
    left = oracle.bearing(W, H, -0.5, 40)
    right = oracle.bearing(W, H, W - 0.5, 40)
    np.testing.assert_allclose(left, right, atol=1e-12)
    # a direction a quarter pixel past the last column's right edge comes back
    # a quarter pixel into the first column
    uc, _ = oracle.project(W, H, oracle.bearing(W, H, W - 0.25, 40))
    assert abs(uc - (-0.25)) < 1e-9


def _rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def test_relative_pose_is_composition():
    """rel(r -> s) applied to pose_r(X) equals pose_s(X) for any world point X."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        Rr, Rs = _rand_rot(rng), _rand_rot(rng)
        tr, ts = rng.normal(size=3), rng.normal(size=3)
        R, t = oracle.rel_pose(Rr, tr, Rs, ts)
        X = rng.normal(size=(10, 3))
        lhs = (R @ (Rr @ X.T + tr[:, None]) + t[:, None]).T
        rhs = (Rs @ X.T + ts[:, None]).T
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_bilinear_sampling():
    rng = np.random.default_rng(2)
    H, W = 6, 10
    img = rng.uniform(0, 1, size=(H, W))
    # integer coordinates return the pixel
    for v in range(H):
        for u in range(W):
            assert oracle.sample(img, u, v) == img[v, u]
    # linear image is reproduced exactly away from the seam and the clamped rows
    lin = 0.01 * np.arange(W)[None, :] + 0.05 * np.arange(H)[:, None] + 0.1
    for uc, vc in [(2.25, 1.5), (7.9, 3.01), (0.5, 4.75)]:
        assert abs(oracle.sample(lin, uc, vc) - (0.01 * uc + 0.05 * vc + 0.1)) < 1e-12
    # the seam: halfway between the last and the first column
    assert abs(oracle.sample(img, W - 0.5, 2) - 0.5 * (img[2, W - 1] + img[2, 0])) < 1e-12
    assert abs(oracle.sample(img, -0.25, 2) - (0.25 * img[2, W - 1] + 0.75 * img[2, 0])) < 1e-12
    # latitude is clamped above the first and below the last row
    assert abs(oracle.sample(img, 3, -0.5) - img[0, 3]) < 1e-12
    assert abs(oracle.sample(img, 3, H - 0.5) - img[H - 1, 3]) < 1e-12


def test_uint8_is_dn_over_255():
    img = np.array([[0, 255], [51, 102]], dtype=np.uint8)
    assert oracle.sample(img, 0, 1) == 51 / 255
    assert oracle.sample(img, 1, 0) == 1.0
