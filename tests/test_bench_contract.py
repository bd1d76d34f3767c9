"""bench.py's reference arm keeps the JSON-line contract (CPU only).

`bench.py --impl reference` times the FP64 oracle on the host cores and
prints one JSON line with the same metric, unit and config as the GPU arm,
plus `impl`, `cpu_baseline` and an `e2e` object without host-device bytes.
Here the workload is swapped for a tiny render so the check takes a second.
"""
import argparse
import contextlib
import io
import json

import bench
import scenes


def _tiny_workload(seed_scene=1001):
    traj = scenes.trajectory(11, seed=2000)
    scene = scenes.Scene(seed=seed_scene)
    scene.objects = scenes.place_objects(seed_scene + 77, [c for _, _, c in traj], n=20)
    frames = []
    for (R, t, C) in traj:
        img, rg = scene.render(R, t, 64, 32, with_range=True)
        frames.append(scenes.Frame(R, t, C, scenes.quantise_u8(img), rg))
    params = dict(d_min=0.3, d_max=10.0, patch_w=11, patch_stride=2, iterations=bench.ITERS, best_k=3,
                  sigma_color=0.2, sigma_space=3.0, n_refine=6, neighbor_table=0, seed=42, keyframe_id=5)
    return frames, params


def test_reference_arm_prints_one_contract_line(monkeypatch):
    monkeypatch.setattr(bench, "make_workload", _tiny_workload)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(steps=2, warmup=1))
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["n_gpus"], d["steps"], d["warmup"]) == (bench.METRIC, "keyframes/s", 1, 2, 1)
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and isinstance(d["dtype"], str)
    assert d["value"] > 0
    # a step is the bounded sample: its wall time is ms_per_step, and the value comes
    # from the keyframe time the sample scales to
    cb = d["cpu_baseline"]
    assert abs(d["ms_per_step"] - 1e3 * cb["sample_s_per_step"]) < 1e-6 * d["ms_per_step"]
    assert abs(cb["keyframe_s_scaled"] - 1.0 / d["value"]) < 1e-6 * cb["keyframe_s_scaled"]
    assert d["config"] == bench.keyframe_config(1) and "workload" in d["config"] and "model" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == dict(value=d["value"], unit=d["unit"], h2d_bytes_per_step=0, d2h_bytes_per_step=0)


def test_reference_arm_is_silent_off_rank_zero(monkeypatch):
    monkeypatch.setattr(bench, "make_workload", _tiny_workload)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    assert buf.getvalue().strip() == ""
