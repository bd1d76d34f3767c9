"""View Filter, point-cloud fusion and completeness on the GPU vs the oracle.

The GPU computes in FP32 and the oracle in FP64, and all three results are
decided by floating-point comparisons (angle bounds, voxel faces, pixel
boundaries). Both sides must agree exactly wherever the oracle's decision is
clear of its threshold; the few decisions within rounding distance bound the
allowed difference in counts.
"""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_16266_gb300 as pm
    return pm


def _bearing(W, H):
    u, v = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    lon = 2 * np.pi * u / W - np.pi
    lat = np.pi / 2 - np.pi * v / H
    return np.stack([np.cos(lat) * np.sin(lon), -np.sin(lat), np.cos(lat) * np.cos(lon)], -1)


@pytest.fixture(scope="module")
def walk():
    W, H = 192, 96
    traj = scenes.trajectory(6, seed=2000)
    scene = scenes.Scene(seed=1001)
    scene.objects = scenes.place_objects(1078, [c for _, _, c in traj], n=20)
    out = []
    for (R, t, C) in traj:
        _, rg = scene.render(R, t, W, H, ss=1)
        out.append(((R, t), rg, C))
    return out


def _shared_points(walk, a, b, n=4000, seed=0):
    """Ground-truth surface points of keyframe a that keyframe b also sees."""
    (Ra, ta), rga, Ca = walk[a]
    (Rb, tb), rgb, Cb = walk[b]
    H, W = rga.shape
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, W * H, n)
    X = Ca + (rga.reshape(-1)[idx, None] * _bearing(W, H).reshape(-1, 3)[idx]) @ Ra
    Y = X @ Rb.T + tb
    dist = np.linalg.norm(Y, axis=1)
    lon = np.arctan2(Y[:, 0], Y[:, 2])
    lat = np.arctan2(-Y[:, 1], np.hypot(Y[:, 0], Y[:, 2]))
    u = np.floor(W * (lon + np.pi) / (2 * np.pi)).astype(int) % W
    v = np.clip(np.floor(H * (np.pi / 2 - lat) / np.pi).astype(int), 0, H - 1)
    seen = np.abs(rgb[v, u] - dist) < 0.02 * dist
    return X[seen]


def test_view_filter_matches_oracle(pm, walk):
    import torch
    for a, b in ((0, 1), (0, 3), (1, 5)):
        pts = _shared_points(walk, a, b, seed=a * 10 + b)
        pa, pb = walk[a][0], walk[b][0]
        pts32 = pts.astype(np.float32)
        acc_o, frac_o, th, flags_o = oracle.view_filter(pa, pb, pts32.astype(np.float64))
        clear = (np.abs(th - 6.0) > 1e-3) & (np.abs(th - 60.0) > 1e-3)
        with pm.Context(0) as ctx:
            flags = torch.zeros(len(pts), dtype=torch.uint8, device="cuda")
            acc, frac, _ = pm.pmsp_view_filter(ctx, pa, pb, torch.from_numpy(pts32).cuda(), in_range=flags)
            flags = flags.cpu().numpy().astype(bool)
            hflags = np.zeros(len(pts), np.uint8)
            acc_h, frac_h, _ = pm.pmsp_view_filter(ctx, pa, pb, pts32, in_range=hflags)
        assert np.array_equal(flags[clear], flags_o[clear])
        assert abs(frac - frac_o) <= np.sum(~clear) / len(pts) + 1e-12
        if abs(frac_o - 0.2) > np.sum(~clear) / len(pts):
            assert acc == acc_o
        assert (acc_h, frac_h) == (acc, frac) and np.array_equal(hflags.astype(bool), flags)
        print(f"keyframes {a},{b}: {len(pts)} points, share in range {frac:.3f}, accepted {acc}")


def test_view_filter_bounds_exact(pm):
    b = 1.0
    A = (np.eye(3), np.array([b / 2, 0, 0]))    # centre (-b/2, 0, 0)
    B = (np.eye(3), np.array([-b / 2, 0, 0]))   # centre (b/2, 0, 0)
    h_of = lambda deg: b / (2 * np.tan(np.radians(deg) / 2))
    inside, outside = [0, 0, h_of(30.0)], [0, 0, h_of(3.0)]
    with pm.Context(0) as ctx:
        for k, want in ((20, False), (21, True)):
            pts = np.array([inside] * k + [outside] * (100 - k), np.float32)
            acc, frac, _ = pm.pmsp_view_filter(ctx, A, B, pts)
            assert frac == k / 100 and acc == want
        acc, frac, _ = pm.pmsp_view_filter(ctx, A, B, np.zeros((0, 3), np.float32))
        assert frac == 0.0 and not acc


def _fuse_both(pm, walk, ks, voxel):
    import torch
    depths = [walk[k][1].astype(np.float32) for k in ks]
    poses = [walk[k][0] for k in ks]
    opts, osrc, margin = oracle.fuse([d.astype(np.float64) for d in depths], poses, voxel)
    with pm.Context(0) as ctx:
        gpts, gsrc, cnt = pm.pmsp_fuse(ctx, [torch.from_numpy(d).cuda() for d in depths], poses, voxel)
        gpts, gsrc = gpts.cpu().numpy(), gsrc.cpu().numpy()
        hpts, hsrc, hcnt = pm.pmsp_fuse(ctx, depths, poses, voxel)
        gpts2, gsrc2, _ = pm.pmsp_fuse(ctx, [torch.from_numpy(d).cuda() for d in depths], poses, voxel)
        gsrc2 = gsrc2.cpu().numpy()
    return depths, poses, (opts, osrc, margin), (gpts, gsrc, cnt), (hpts, hsrc, hcnt), gsrc2


def test_fuse_matches_oracle(pm, walk):
    ks, voxel = (1, 2, 3), 0.0437
    depths, poses, (opts, osrc, margin), (gpts, gsrc, cnt), (hpts, hsrc, hcnt), gsrc2 = _fuse_both(pm, walk, ks, voxel)
    unclear = int(np.sum((margin >= 0) & (margin < 1e-4)))
    assert cnt == len(gsrc) and abs(cnt - len(osrc)) <= unclear
    assert np.all(np.diff(gsrc) > 0)                     # written in (keyframe, pixel) order
    assert np.array_equal(gsrc, gsrc2)                   # independent of thread timing
    assert hcnt == cnt and np.array_equal(hsrc, gsrc) and np.array_equal(hpts, gpts)
    diff = set(gsrc.tolist()) ^ set(osrc.tolist())
    assert len(diff) <= 4 * unclear + 0, (len(diff), unclear)
    # the kept points themselves: FP32 lifts of the same pixels
    o_by_src = dict(zip(osrc.tolist(), opts))
    common = [i for i, s in enumerate(gsrc.tolist()) if s in o_by_src]
    ref = np.array([o_by_src[s] for s in gsrc[common].tolist()])
    assert np.max(np.abs(gpts[common] - ref)) < 2e-5 * 10
    print(f"fused {len(ks)} keyframes: {cnt} voxels (oracle {len(osrc)}), {unclear} points within 1e-4 voxel of a face")


def test_fuse_capacity_and_errors(pm, walk):
    import torch
    d = torch.from_numpy(walk[0][1].astype(np.float32)).cuda()
    with pm.Context(0) as ctx:
        pts, src, cnt = pm.pmsp_fuse(ctx, [d], [walk[0][0]], 0.05)
        p2, s2, c2 = pm.pmsp_fuse(ctx, [d], [walk[0][0]], 0.05, cap=100)
        assert c2 == cnt and len(s2) == 100 and np.array_equal(s2.cpu().numpy(), src[:100].cpu().numpy())
        for bad in (dict(voxel=0.0), dict(voxel=1e-9)):
            with pytest.raises(pm.PmspError) as e:
                pm.pmsp_fuse(ctx, [d], [walk[0][0]], **bad)
            assert e.value.code == pm.PMSP_EINVAL


def test_completeness_matches_oracle(pm, walk):
    import torch
    ks = (1, 2, 3)
    depths = [walk[k][1].astype(np.float32) for k in ks]
    poses = [walk[k][0] for k in ks]
    with pm.Context(0) as ctx:
        pts, _, _ = pm.pmsp_fuse(ctx, [torch.from_numpy(d).cuda() for d in depths], poses, 0.02)
        for k in (0, 2, 4):
            hit = torch.zeros((360, 720), dtype=torch.uint8, device="cuda")
            c, _ = pm.pmsp_completeness(ctx, pts, walk[k][0], 720, 360, hit=hit)
            hit = hit.cpu().numpy().astype(bool)
            P = pts.cpu().numpy().astype(np.float64)
            co, ho, mg = oracle.completeness(P, walk[k][0], 720, 360)
            unclear = int(np.sum(mg < 1e-3))
            assert np.sum(hit != ho) <= 2 * unclear
            assert abs(c - co) <= unclear / (720 * 360) + 1e-12
            hh = np.zeros((360, 720), np.uint8)
            ch, _ = pm.pmsp_completeness(ctx, P.astype(np.float32), walk[k][0], 720, 360, hit=hh)
            assert ch == c and np.array_equal(hh.astype(bool), hit)
            print(f"keyframe {k}: completeness {c:.4f} (oracle {co:.4f}), {unclear} points near a pixel edge")


def test_view_filter_and_completeness_errors(pm):
    pts = np.zeros((4, 3), np.float32)
    pose = (np.eye(3), np.zeros(3))
    with pm.Context(0) as ctx:
        for kw in (dict(min_deg=30.0, max_deg=10.0), dict(max_deg=181.0), dict(min_frac=1.5), dict(min_deg=-1.0)):
            with pytest.raises(pm.PmspError) as e:
                pm.pmsp_view_filter(ctx, pose, pose, pts, **kw)
            assert e.value.code == pm.PMSP_EINVAL
        with pytest.raises(pm.PmspError) as e:
            pm.pmsp_completeness(ctx, pts, pose, 0, 10)
        assert e.value.code == pm.PMSP_EINVAL
