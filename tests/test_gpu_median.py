"""Median post-filter on the GPU vs the oracle (Sec. III-C, item 2).

Selection is exact and the removal decision is FP32 on both sides, so the
filtered maps must be identical bit for bit: on maps with holes of several
sizes (ragged tiles, a panorama narrower than the window, every radius), on a
densified map, at 1920x960, and through host buffers.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_16266_gb300 as pm
    return pm


def _map(W, H, seed, holes=0.2, spikes=0.03):
    rng = np.random.default_rng(seed)
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    d = 2.0 + 0.6 * np.sin(2 * np.pi * u / W) * np.cos(np.pi * v / H) + 0.02 * rng.standard_normal((H, W))
    d = np.where(rng.random((H, W)) < spikes, d * rng.uniform(0.5, 1.6, (H, W)), d)
    d[rng.random((H, W)) < holes] = 0.0
    return d.astype(np.float32)


def _gpu(pm, ctx, d, r, tau):
    import torch
    t = torch.from_numpy(d).cuda()
    return pm.pmsp_median_filter(ctx, t, r, tau).cpu().numpy()


@pytest.mark.parametrize("W,H,r", [(64, 32, 2), (100, 37, 2), (8, 4, 3), (6, 3, 2), (250, 123, 1), (96, 40, 3)])
def test_median_bit_exact(pm, W, H, r):
    d = _map(W, H, seed=W * 7 + H + r)
    want, _ = oracle.median_filter(d.astype(np.float64), r, 0.05)
    with pm.Context(0) as ctx:
        got = _gpu(pm, ctx, d, r, 0.05)
    assert np.array_equal(got, want.astype(np.float32))
    if W >= 64:  # smooth surface with spikes: the spikes go, little else
        assert 0 < np.mean((d > 0) & (got == 0)) < 0.2


def test_median_on_densified_map(pm):
    import scenes
    prob = scenes.config0()
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with pm.Context(0) as ctx:
        m = pm.pmsp_densify(ctx, dev(prob.ref.image), (prob.ref.R, prob.ref.t), [dev(f.image) for f in prob.srcs],
                            [(f.R, f.t) for f in prob.srcs], prob.params)
        d = m.depth.cpu().numpy()
        got = _gpu(pm, ctx, d, 2, 0.05)
    want, _ = oracle.median_filter(d.astype(np.float64), 2, 0.05)
    assert np.array_equal(got, want.astype(np.float32))


def test_median_full_size_and_host_buffers(pm):
    d = _map(1920, 960, seed=5)
    want, _ = oracle.median_filter(d.astype(np.float64), 2, 0.05)
    with pm.Context(0) as ctx:
        got = _gpu(pm, ctx, d, 2, 0.05)
        host = pm.pmsp_median_filter(ctx, d, 2, 0.05)
    assert np.array_equal(got, want.astype(np.float32))
    assert np.array_equal(host, got)


def test_median_errors(pm):
    import torch
    d = torch.ones((8, 16), device="cuda")
    with pm.Context(0) as ctx:
        for kw in (dict(radius=0), dict(radius=4), dict(tau=0.0)):
            with pytest.raises(pm.PmspError) as e:
                pm.pmsp_median_filter(ctx, d, **kw)
            assert e.value.code == pm.PMSP_EINVAL
        with pytest.raises(pm.PmspError) as e:
            pm.pmsp_median_filter(ctx, d, out=d)
        assert e.value.code == pm.PMSP_EINVAL
