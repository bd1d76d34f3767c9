"""Pins for the oracle's matching cost (bilaterally weighted NCC, best-k).

The paper cites PatchMatch stereo (Bleyer et al.) and Gipuma (Galliani et
al.) for the patch cost without restating it (Sec. I, Sec. III-C). The pins:

* pure rotation about the vertical axis by k pixels: every plane maps each
  patch sample exactly onto the source pixel k columns over, so the source
  patch is a plain array slice of the source image; the per-view cost then
  equals 1 - numpy.corrcoef (or the aweights-weighted numpy.cov ratio) of
  two array slices, and a rolled copy of the reference gives cost 0;
* affine intensity changes leave the cost unchanged, a negated source gives
  cost 2 for a view, best-k is the mean of the k smallest known view costs;
* with zero translation the cost does not depend on the range;
* ground-truth planes of a rendered room score far below random planes, and
  where the wall is seen obliquely they beat the fronto-parallel plane at the
  same range (the slant acts only through each sample's range along its ray).
"""
import math

import numpy as np
import pytest

import oracle
import scenes

W, H = 64, 32


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def _texture(seed, shape=(H, W)):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=shape)


def _problem(ref, srcs_k, **params):
    """Sources given as (image, k): pose = yaw by 2*pi*k/W, no translation."""
    I3, z = np.eye(3), np.zeros(3)
    poses = [(_rot_y(2 * math.pi * k / W), z) for _, k in srcs_k]
    return oracle.Problem(ref, (I3, z), [s for s, _ in srcs_k], poses, **params)


def _patch(img, u, v, offs, shift=0):
    rows = [min(max(v + oy, 0), H - 1) for oy in offs for ox in offs]
    cols = [(u + ox + shift) % W for oy in offs for ox in offs]
    return img[rows, cols]


def _plane(u, v, d, rng):
    r = oracle.bearing(W, H, u, v)
    n = -r + 0.3 * rng.normal(size=3)
    n /= np.linalg.norm(n)
    if n @ r > -0.5:
        n = -r
    return d, n


PIXELS = [(0, 0), (W - 1, 5), (10, 16), (33, H - 1), (W // 2, H // 2), (1, 30)]


@pytest.mark.parametrize("k", [0, 3, -5, W // 2])
def test_rolled_reference_costs_zero(k):
    ref = _texture(10)
    pb = _problem(ref, [(np.roll(ref, k, axis=1), k)], patch_w=7, patch_stride=1, best_k=1)
    rng = np.random.default_rng(11)
    for (u, v) in PIXELS:
        d, n = _plane(u, v, rng.uniform(0.5, 5), rng)
        assert pb.cost(u, v, d, n) < 1e-9


@pytest.mark.parametrize("patch_w,stride", [(7, 1), (11, 2), (5, 2)])
def test_unweighted_cost_is_one_minus_corrcoef(patch_w, stride):
    ref, src = _texture(20), _texture(21)
    k = 7
    pb = _problem(ref, [(src, k)], patch_w=patch_w, patch_stride=stride, best_k=1)
    r = (patch_w - 1) // 2
    offs = list(range(-r, r + 1, stride))
    rng = np.random.default_rng(22)
    for (u, v) in PIXELS:
        d, n = _plane(u, v, rng.uniform(0.5, 5), rng)
        I = _patch(ref, u, v, offs)
        J = _patch(src, u, v, offs, shift=k)
        expect = 1.0 - np.corrcoef(I, J)[0, 1]
        assert abs(pb.cost(u, v, d, n) - expect) < 1e-10


def test_weighted_cost_is_weighted_pearson():
    ref, src = _texture(30), _texture(31)
    k, sc, ss = -4, 0.2, 3.0
    pb = _problem(ref, [(src, k)], patch_w=11, patch_stride=2, best_k=1, sigma_color=sc, sigma_space=ss)
    offs = list(range(-5, 6, 2))
    rng = np.random.default_rng(32)
    for (u, v) in PIXELS:
        d, n = _plane(u, v, rng.uniform(0.5, 5), rng)
        I = _patch(ref, u, v, offs)
        J = _patch(src, u, v, offs, shift=k)
        o2 = np.array([ox * ox + oy * oy for oy in offs for ox in offs], dtype=float)
        w = np.exp(-(I - ref[v, u]) ** 2 / (2 * sc * sc) - o2 / (2 * ss * ss))
        C = np.cov(I, J, aweights=w)
        expect = 1.0 - C[0, 1] / math.sqrt(C[0, 0] * C[1, 1])
        assert abs(pb.cost(u, v, d, n) - expect) < 1e-10
        # without the weights the value differs (the weights are in effect)
        assert abs(expect - (1 - np.corrcoef(I, J)[0, 1])) > 1e-6


def test_affine_invariance_and_negation():
    ref, src = _texture(40), _texture(41)
    k = 9
    base = _problem(ref, [(src, k)], patch_w=7, patch_stride=1, best_k=1)
    aff = _problem(ref, [(0.5 * src + 0.2, k)], patch_w=7, patch_stride=1, best_k=1)
    neg = _problem(ref, [(np.roll(1.0 - ref, k, axis=1), k)], patch_w=7, patch_stride=1, best_k=1)
    rng = np.random.default_rng(42)
    for (u, v) in PIXELS:
        d, n = _plane(u, v, 2.0, rng)
        assert abs(base.cost(u, v, d, n) - aff.cost(u, v, d, n)) < 1e-10
        assert abs(neg.cost(u, v, d, n) - 2.0) < 1e-10


@pytest.mark.parametrize("best_k", [1, 2, 3])
def test_best_k_mean_of_smallest(best_k):
    ref, other = _texture(50), _texture(51)
    views = [(np.roll(1.0 - ref, 2, axis=1), 2),      # cost 2
             (np.roll(ref, -3, axis=1), -3),          # cost 0
             (other, 5)]                              # cost 1 - corrcoef
    pb = _problem(ref, views, patch_w=7, patch_stride=1, best_k=best_k)
    offs = list(range(-3, 4))
    rng = np.random.default_rng(52)
    for (u, v) in PIXELS:
        d, n = _plane(u, v, 1.5, rng)
        c = 1.0 - np.corrcoef(_patch(ref, u, v, offs), _patch(other, u, v, offs, shift=5))[0, 1]
        expect = {1: 0.0, 2: c / 2, 3: (2 + c) / 3}[best_k]
        assert abs(pb.cost(u, v, d, n) - expect) < 1e-10


def test_flat_source_and_invalid_plane_cost_two():
    ref = _texture(60)
    flat = _problem(ref, [(np.full((H, W), 0.4), 0)], patch_w=7, patch_stride=1, best_k=1)
    u, v = 20, 12
    r = oracle.bearing(W, H, u, v)
    assert flat.cost(u, v, 2.0, -r) == 2.0
    pb = _problem(ref, [(np.roll(ref, 1, axis=1), 1)], patch_w=7, patch_stride=1, best_k=1)
    # grazing plane: faces pixel p but some patch rays hit it from behind
    t = np.cross(r, [0, 1, 0])
    t /= np.linalg.norm(t)
    n = -0.01 * r + t
    n /= np.linalg.norm(n)
    assert n @ r < 0
    assert pb.cost(u, v, 2.0, n) == 2.0


def test_zero_translation_cost_independent_of_range():
    ref, src = _texture(70), _texture(71)
    rng = np.random.default_rng(72)
    R = _rot_y(0.37) @ np.array([[1, 0, 0], [0, math.cos(0.2), -math.sin(0.2)], [0, math.sin(0.2), math.cos(0.2)]])
    pb = oracle.Problem(ref, (np.eye(3), np.zeros(3)), [src], [(R, np.zeros(3))], patch_w=7,
                        patch_stride=1, best_k=1)
    for (u, v) in PIXELS:
        _, n = _plane(u, v, 1.0, rng)
        c1, c2 = pb.cost(u, v, 0.4, n), pb.cost(u, v, 7.0, n)
        assert abs(c1 - c2) < 1e-9


def _wall_normals_cam(prob, depth):
    """Camera-frame normals of the room wall hit by every pixel's centre ray."""
    Hh, Ww = depth.shape
    R, C = prob.ref.R, prob.ref.centre
    lo, hi = prob.scene.lo, prob.scene.hi
    n = np.zeros((3, Hh, Ww))
    for v in range(Hh):
        for u in range(Ww):
            r = oracle.bearing(Ww, Hh, u, v)
            X = C + depth[v, u] * (R.T @ r)
            nw = np.zeros(3)
            a = int(np.argmin(np.minimum(np.abs(X - lo), np.abs(X - hi))))
            nw[a] = 1.0 if abs(X[a] - lo[a]) < abs(X[a] - hi[a]) else -1.0
            n[:, v, u] = R @ nw
    return n


def test_ground_truth_planes_beat_random_planes():
    prob = scenes.config0()
    pb = oracle.Problem.from_scene(prob)
    gt = prob.ref.range
    n_gt = _wall_normals_cam(prob, gt)
    c_gt = pb.cost_map(gt, n_gt)
    _, _, c_init = pb.init()
    assert np.mean(c_gt < np.median(c_init)) > 0.9
    assert np.mean(c_gt < 0.1) > 0.8
    # a planted transposition of the source rotation must destroy the fit
    bad = oracle.Problem(prob.ref.image, (prob.ref.R, prob.ref.t), [f.image for f in prob.srcs],
                         [(f.R.T, f.t) for f in prob.srcs], **prob.params)
    c_bad = bad.cost_map(gt, n_gt)
    assert np.mean(c_bad < 0.1) < 0.5


def test_slanted_ground_truth_planes_beat_fronto_parallel_planes():
    """A patch on a wall seen obliquely is explained by the wall's own plane, not by
    the plane facing the camera at the same range: where the incidence cosine
    |n . r_p| is at most 0.9, the ground-truth plane scores lower than the
    fronto-parallel one (normal -r_p) on most pixels. The slant enters only through
    the range of each patch sample along its own ray, t_q = d (n . r_p) / (n . r_q)."""
    prob = scenes.config0()
    pb = oracle.Problem.from_scene(prob)
    gt = prob.ref.range
    n_gt = _wall_normals_cam(prob, gt)
    Hh, Ww = gt.shape
    r = np.stack([oracle.bearing(Ww, Hh, u, v) for v in range(Hh) for u in range(Ww)])
    r = r.reshape(Hh, Ww, 3).transpose(2, 0, 1)
    slanted = -np.sum(n_gt * r, 0) <= 0.9
    assert slanted.sum() > 0.3 * gt.size
    c_gt = pb.cost_map(gt, n_gt)
    c_fp = pb.cost_map(gt, -r)
    assert np.mean(c_gt[slanted] < c_fp[slanted]) > 0.75
