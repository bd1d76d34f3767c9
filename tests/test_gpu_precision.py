"""Precision forms: images stored as FP16 or uint8, FP32 arithmetic on the GPU.

The 8-bit texture with N(0, 2 DN) noise of the 3840x1920 workload is
rendered at 768x384 (the FP64 oracle finishes it in seconds) with 8 sources.
For each storage form the GPU maps are compared with the FP64 oracle run on
the same stored values, and both are compared with the ground-truth range.
FP16 holds the noisy intensities to 11 bits, uint8 rounds them to whole DN,
so the two forms see slightly different inputs; their accuracy against
ground truth must be the same within a small margin.
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def forms():
    return {fmt: scenes.config2(W=768, H=384, fmt=fmt) for fmt in ("f16", "u8")}


def test_each_form_matches_fp64_oracle_and_ground_truth(pm, forms):
    acc = {}
    with pm.Context(0) as ctx:
        for fmt, prob in forms.items():
            args = (_dev(prob.ref.image), (prob.ref.R, prob.ref.t), [_dev(f.image) for f in prob.srcs],
                    [(f.R, f.t) for f in prob.srcs])
            gd, _, gc = (a.astype(np.float64) for a in pm.pmsp_densify(ctx, *args, prob.params).numpy())
            od, _, oc = oracle.Problem.from_scene(prob).densify()
            gt = prob.ref.range
            depth_parity = np.mean(np.abs(gd - od) / od <= 5e-3)
            cost_parity = np.mean(np.abs(gc - oc) <= 1e-4)
            acc[fmt] = dict(gpu=np.mean(np.abs(gd - gt) / gt < 0.05), oracle=np.mean(np.abs(od - gt) / gt < 0.05),
                            gpu_1=np.mean(np.abs(gd - gt) / gt < 0.01), parity=depth_parity)
            print(f"{fmt}: depth parity {depth_parity:.4f} cost parity {cost_parity:.4f} "
                  f"GT<5%: gpu {acc[fmt]['gpu']:.4f} oracle {acc[fmt]['oracle']:.4f} GT<1%: gpu {acc[fmt]['gpu_1']:.4f}")
            assert depth_parity >= 0.995 and cost_parity >= 0.995
            assert abs(acc[fmt]["gpu"] - acc[fmt]["oracle"]) < 0.01
    assert abs(acc["f16"]["gpu"] - acc["u8"]["gpu"]) < 0.02
