"""The no-allocation batch entry point (pmsp_densify_batch_noalloc).

Callers that cannot allocate device memory when they densify (frameworks
that own all device memory, real-time threads, code running while a stream
is recorded) use this entry point; its batch state lives in a fixed
__device__ array instead of allocated buffers. Its maps must agree with the
ordinary batched entry point within the parity tolerances (it reads sources
with plain loads instead of texture gathers, so uint8 conversion may differ
in the last bit), on two calls in a row: the second call reuses the array
the first one left behind. Two of the keyframes (the plain-load uint8 and FP32
fetches) are also held to the FP64 oracle's whole densification at the same bar.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_batched_entry_point_twice():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_16266_gb300 as pm

    p1 = scenes.config1(W=384, H=192)
    p2 = scenes.trajectory_problem(250, 132, 3, seed_scene=1010)
    p2.params = dict(d_min=0.3, d_max=10.0, patch_w=9, patch_stride=3, iterations=3, best_k=2, sigma_color=0.15,
                     sigma_space=4.0, n_refine=6, neighbor_table=1, seed=5, keyframe_id=77)
    p3 = scenes.trajectory_problem(256, 128, 4, seed_scene=1012, fmt="f16")
    p3.params = dict(p1.params, iterations=4, keyframe_id=9)
    p4 = scenes.trajectory_problem(192, 96, 3, seed_scene=1014, fmt="f32")
    p4.params = dict(p1.params, iterations=3, best_k=2, keyframe_id=4)
    probs = [p1, p2, p3, p4]
    args = [(_dev(p.ref.image), (p.ref.R, p.ref.t), [_dev(f.image) for f in p.srcs], [(f.R, f.t) for f in p.srcs])
            for p in probs]
    with pm.Context(0) as ctx:
        want = [o.numpy() for o in pm.pmsp_densify_batch(ctx, pm.Batch([(*a, p.params, None)
                                                                       for a, p in zip(args, probs)]))]
        for call in range(2):
            got = pm.pmsp_densify_batch_noalloc(ctx, pm.Batch([(*a, p.params, None) for a, p in zip(args, probs)]))
            pm.pmsp_sync(ctx)
            for (wd, wn, wc), o in zip(want, got):
                gd, gn, gc = o.numpy()
                assert np.mean(np.abs(gd - wd) / wd <= 5e-3) >= 0.995, call
                assert np.mean(np.abs(gc - wc) <= 1e-4) >= 0.995, call
            if call == 0:
                for k in (1, 3):
                    od, on, oc = oracle.Problem.from_scene(probs[k]).densify()
                    gd, gn, gc = (a.astype(np.float64) for a in got[k].numpy())
                    assert np.mean(np.abs(gd - od) / od <= 5e-3) >= 0.995, k
                    assert np.mean(np.abs(gc - oc) <= 1e-4) >= 0.995, k
        # a batch above the stated limit is refused, and nothing is run
        big = pm.Batch([(*args[2], probs[2].params, None)] * (pm.PMSP_NOALLOC_MAX_ITEMS + 1))
        with pytest.raises(pm.PmspError) as e:
            pm.pmsp_densify_batch_noalloc(ctx, big)
        assert e.value.code == pm.PMSP_EINVAL


def test_noalloc_recorded_in_a_graph_replays_the_same_maps():
    """A call made while the context's stream is being recorded puts all of its
    work into the graph, its descriptors included (nothing is read from host
    memory at replay): every replay gives the maps of a direct call, bit for bit."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_16266_gb300 as pm

    p = scenes.config1(W=256, H=128)
    p.params = dict(p.params, iterations=3)
    a = (_dev(p.ref.image), (p.ref.R, p.ref.t), [_dev(f.image) for f in p.srcs], [(f.R, f.t) for f in p.srcs])
    s = torch.cuda.Stream()
    with pm.Context(0, stream=s) as ctx:
        batch = pm.Batch([(*a, p.params, None)])
        pm.pmsp_densify_batch_noalloc(ctx, batch)   # the first call on a device, outside any capture
        pm.pmsp_sync(ctx)
        want = [x.copy() for x in batch.outs[0].numpy()]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            pm.pmsp_densify_batch_noalloc(ctx, batch)
        out = batch.outs[0]
        for x in (out.depth, out.normal, out.cost):
            x.zero_()
        for _ in range(2):
            g.replay()
            torch.cuda.synchronize()
            for w, x in zip(want, out.numpy()):
                assert np.array_equal(w, x)
            out.depth.zero_()
