"""The parameters the paper prints (tests/golden/paper_parameters.txt) are the
defaults of both the oracle and the C-ABI binding, and the View Filter's bounds
behave as Eq. 1 states them on the oracle.
"""
import inspect
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, value = line.split()
                vals[name] = float(value)
    return vals


def _defaults(fn):
    return {k: p.default for k, p in inspect.signature(fn).parameters.items()
            if p.default is not inspect.Parameter.empty}


def test_defaults_are_the_papers():
    import paper_2211_16266_gb300 as pm
    g = _golden()
    for fn in (oracle.view_filter, pm.pmsp_view_filter):
        d = _defaults(fn)
        assert (d["min_deg"], d["max_deg"], d["min_frac"]) == (
            g["view_filter_min_deg"], g["view_filter_max_deg"], g["view_filter_min_frac"])
    for fn in (oracle.completeness, pm.pmsp_completeness):
        d = _defaults(fn)
        assert (d["W"], d["H"]) == (g["completeness_width"], g["completeness_height"])


def test_printed_view_filter_bounds_on_the_oracle():
    """Two centres a baseline b apart see a point at height h on their bisector under
    2 atan(b / 2h); the angles just inside the printed bounds count, those just outside
    do not, and acceptance needs more than the printed share."""
    g = _golden()
    b = 1.0
    A = (np.eye(3), np.array([b / 2, 0, 0]))
    B = (np.eye(3), np.array([-b / 2, 0, 0]))
    h_of = lambda deg: b / (2 * np.tan(np.radians(deg) / 2))
    lo, hi = g["view_filter_min_deg"], g["view_filter_max_deg"]
    degs = [lo - 0.01, lo + 0.01, 0.5 * (lo + hi), hi - 0.01, hi + 0.01]
    pts = np.array([[0, 0, h_of(d)] for d in degs])
    _, _, theta, flags = oracle.view_filter(A, B, pts)
    assert np.allclose(theta, degs, atol=1e-9)
    assert flags.tolist() == [False, True, True, True, False]
    n = 100
    k = int(round(g["view_filter_min_frac"] * n))
    inside, outside = [0, 0, h_of(0.5 * (lo + hi))], [0, 0, h_of(lo / 2)]
    for kk, want in ((k, False), (k + 1, True)):
        acc, frac, _, _ = oracle.view_filter(A, B, np.array([inside] * kk + [outside] * (n - kk)))
        assert frac == kk / n and acc == want
