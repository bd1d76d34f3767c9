"""Pins for the oracle's View Filter (Sec. III-A, Eq. 1).

The parallax angle at a point is checked against closed forms that do not
use the oracle's formula: the isosceles configuration (a point on the
perpendicular bisector of the baseline sees it under 2 atan(b / 2h)), the
law of cosines on the triangle's side lengths, collinear points (0 and 180
degrees), and invariance under rigid motion and scale of the whole scene;
the acceptance rule is checked at its 20 % boundary and at the angle bounds.
"""
import numpy as np

import oracle


def _pose_at(C, R=np.eye(3)):
    C = np.asarray(C, float)
    return R, -R @ C


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def test_bisector_closed_form():
    b = 0.3
    A, B = _pose_at([-b / 2, 0, 0]), _pose_at([b / 2, 0, 0], _rot([0, 1, 0], 0.4))
    hs = np.array([0.05, 0.2, 0.5, 1.0, 3.0, 10.0])
    pts = np.stack([np.zeros_like(hs), np.zeros_like(hs), hs], 1)
    _, _, th, _ = oracle.view_filter(A, B, pts)
    want = np.degrees(2 * np.arctan(b / (2 * hs)))
    np.testing.assert_allclose(th, want, rtol=0, atol=1e-10)


def test_law_of_cosines_random_points():
    rng = np.random.default_rng(0)
    CA, CB = rng.normal(size=3), rng.normal(size=3)
    A, B = _pose_at(CA, _rot(rng.normal(size=3), 1.0)), _pose_at(CB, _rot(rng.normal(size=3), 2.0))
    pts = rng.normal(size=(200, 3)) * 3
    _, _, th, _ = oracle.view_filter(A, B, pts)
    a = np.linalg.norm(pts - CA, axis=1)
    bb = np.linalg.norm(pts - CB, axis=1)
    c = np.linalg.norm(CA - CB)
    want = np.degrees(np.arccos(np.clip((a * a + bb * bb - c * c) / (2 * a * bb), -1, 1)))
    np.testing.assert_allclose(th, want, atol=1e-7)


def test_collinear_points():
    A, B = _pose_at([0, 0, 0]), _pose_at([1, 0, 0])
    pts = np.array([[2.0, 0, 0], [-3.0, 0, 0], [0.5, 0, 0]])
    _, _, th, flags = oracle.view_filter(A, B, pts)
    np.testing.assert_allclose(th, [0.0, 0.0, 180.0], atol=1e-6)
    assert not flags.any()


def test_point_at_a_camera_centre_counts_out_of_range():
    A, B = _pose_at([0, 0, 0]), _pose_at([1, 0, 0])
    acc, frac, th, flags = oracle.view_filter(A, B, np.array([[0.0, 0, 0], [0.5, 0, 1.0]]))
    assert np.isnan(th[0]) and not flags[0] and flags[1]
    assert frac == 0.5 and acc


def test_rigid_motion_and_scale_invariance():
    rng = np.random.default_rng(1)
    CA, CB = np.array([0.0, 0, 0]), np.array([0.2, 0.05, -0.1])
    pts = rng.normal(size=(300, 3)) * 2
    _, f0, th0, _ = oracle.view_filter(_pose_at(CA), _pose_at(CB), pts)
    Q, s, o = _rot([1, 2, 3], 0.7), 2.5, np.array([4.0, -1, 2])
    T = lambda X: s * (X @ Q.T) + o
    _, f1, th1, _ = oracle.view_filter(_pose_at(T(CA), _rot([0, 0, 1], 1.3)), _pose_at(T(CB)), T(pts))
    np.testing.assert_allclose(th1, th0, atol=1e-9)
    assert f1 == f0


def test_angle_bounds_and_twenty_percent_rule():
    b = 1.0
    A, B = _pose_at([-b / 2, 0, 0]), _pose_at([b / 2, 0, 0])
    h_of = lambda deg: b / (2 * np.tan(np.radians(deg) / 2))
    angles = [5.9, 6.1, 30.0, 59.9, 60.1]
    pts = np.array([[0, 0, h_of(a)] for a in angles])
    _, _, th, flags = oracle.view_filter(A, B, pts)
    assert flags.tolist() == [False, True, True, True, False]
    # 20 of 100 in range: not more than 20 %, rejected; 21 of 100: accepted
    inside, outside = [0, 0, h_of(30.0)], [0, 0, h_of(3.0)]
    for k, want in ((20, False), (21, True)):
        pts = np.array([inside] * k + [outside] * (100 - k))
        acc, frac, _, _ = oracle.view_filter(A, B, pts)
        assert frac == k / 100 and acc == want
