"""Pins for the oracle's median post-filter (Sec. III-C, item 2).

The filter is a plain definition (lower median of the valid ranges in a
seam-wrapped window, removal beyond a relative threshold), so it is pinned
against a library median on fully valid interiors, against brute force on tiny
maps with holes, and by the invariants any median filter has: constants and
monotone ramps survive, an isolated spike is removed, rolling the panorama
rolls the result, and scaling by a power of two scales the medians exactly.
"""
import numpy as np
import pytest

import oracle


def _smooth(W=64, H=32, seed=0):
    rng = np.random.default_rng(seed)
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    d = 2.0 + 0.5 * np.sin(2 * np.pi * u / W) + 0.01 * v + 0.001 * rng.standard_normal((H, W))
    return d.astype(np.float32).astype(np.float64)


def test_constant_map_survives():
    d = np.full((16, 32), 3.25)
    out, med = oracle.median_filter(d, 2, 0.05)
    assert np.array_equal(out, d)
    assert np.array_equal(med, d)


def test_interior_median_matches_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    d = (1.0 + rng.random((24, 40))).astype(np.float32).astype(np.float64)
    _, med = oracle.median_filter(d, 2, 0.05)
    ref = ndimage.median_filter(d, size=5, mode="wrap")
    # 25 valid values: the lower median is the ordinary median; rows 2..H-3 see no row edge
    assert np.array_equal(med[2:-2], ref[2:-2])


def test_brute_force_with_holes_and_edges():
    rng = np.random.default_rng(2)
    H, W, r, tau = 7, 10, 2, 0.05
    d = (1.0 + rng.random((H, W))).astype(np.float32).astype(np.float64)
    d[rng.random((H, W)) < 0.35] = 0.0
    out, med = oracle.median_filter(d, r, tau)
    for v in range(H):
        for u in range(W):
            if d[v, u] <= 0:
                assert out[v, u] == 0 and med[v, u] == 0
                continue
            vals = sorted(d[y, x % W] for y in range(v - r, v + r + 1) if 0 <= y < H
                          for x in range(u - r, u + r + 1) if d[y, x % W] > 0)
            m = vals[(len(vals) - 1) // 2]
            assert med[v, u] == m
            keep = abs(np.float32(d[v, u]) - np.float32(m)) <= np.float32(tau) * np.float32(m)
            assert out[v, u] == (d[v, u] if keep else 0.0)


def test_spike_removed_neighbours_kept():
    d = _smooth()
    d[10, 20] *= 1.5
    out, _ = oracle.median_filter(d, 2, 0.05)
    assert out[10, 20] == 0
    mask = np.ones_like(d, bool)
    mask[10, 20] = False
    assert np.array_equal(out[mask], d[mask])


def test_monotone_ramp_survives():
    H, W = 20, 48
    d = np.tile(1.0 + 0.01 * np.arange(H)[:, None], (1, W))
    out, med = oracle.median_filter(d, 2, 0.05)
    assert np.array_equal(out, d)
    # in the interior the median of a ramp along rows is the centre row
    assert np.array_equal(med[2:-2], d[2:-2])


def test_seam_roll_equivariance():
    d = _smooth(seed=3)
    d[5, 0] *= 1.3
    d[9, 63] *= 0.6
    out, med = oracle.median_filter(d, 2, 0.05)
    for k in (1, 7, 33):
        o2, m2 = oracle.median_filter(np.roll(d, k, axis=1), 2, 0.05)
        assert np.array_equal(o2, np.roll(out, k, axis=1))
        assert np.array_equal(m2, np.roll(med, k, axis=1))
    assert out[5, 0] == 0 and out[9, 63] == 0


def test_power_of_two_scaling():
    d = _smooth(seed=4)
    d[3, 3] *= 1.07
    out, med = oracle.median_filter(d, 2, 0.05)
    o2, m2 = oracle.median_filter(4.0 * d, 2, 0.05)
    assert np.array_equal(m2, 4.0 * med)
    assert np.array_equal(o2 > 0, out > 0)


def test_threshold_is_relative_and_strict():
    # window of 25 ones and a centre at exactly 1 + tau (in float) stays; a hair above goes
    tau = np.float32(0.25)
    d = np.ones((9, 9))
    d[4, 4] = float(np.float32(1.0) + tau)
    out, _ = oracle.median_filter(d, 2, float(tau))
    assert out[4, 4] == d[4, 4]
    d[4, 4] = float(np.nextafter(np.float32(1.0) + tau, np.float32(2.0)))
    out, _ = oracle.median_filter(d, 2, float(tau))
    assert out[4, 4] == 0
