"""The Python binding's argument marshalling, on the CPU (no call crosses into CUDA).

Images become pmsp_image with the array's own row pitch, format and memory
kind (non-contiguous rows are copied first and the copy is kept alive);
poses become row-major FP64 (R, t); parameter dicts override the library's
defaults field by field and unknown names are refused; host maps describe
numpy buffers; a Batch keeps every referenced buffer and lays out the items.
"""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_16266_gb300 as pm
    return pm


def test_images(pm):
    keep = []
    for dtype, fmt in ((np.uint8, pm.PMSP_U8), (np.float16, pm.PMSP_F16), (np.float32, pm.PMSP_F32)):
        a = np.arange(6 * 10, dtype=dtype).reshape(6, 10)
        im = pm.make_image(a, keep)
        assert (im.w, im.h, im.pitch_bytes, im.format, im.memory) == (10, 6, 10 * a.itemsize, fmt, pm.PMSP_HOST)
        assert im.data == a.ctypes.data
    # a row-strided view keeps its pitch: rows are contiguous
    big = np.zeros((6, 16), np.uint8)
    im = pm.make_image(big[:, :10], keep)
    assert (im.w, im.pitch_bytes, im.data) == (10, 16, big.ctypes.data)
    # a column-strided view is copied; the copy is what the struct points to and stays alive
    a = np.arange(40, dtype=np.float32).reshape(4, 10)[:, ::2]
    im = pm.make_image(a, keep)
    assert (im.w, im.h, im.pitch_bytes) == (5, 4, 20)
    assert any(isinstance(k, np.ndarray) and k.ctypes.data == im.data for k in keep)
    got = np.ctypeslib.as_array(ctypes.cast(im.data, ctypes.POINTER(ctypes.c_float)), shape=(4, 5))
    assert np.array_equal(got, a)
    with pytest.raises(KeyError):
        pm.make_image(np.zeros((4, 4), np.int32), keep)


def test_poses_and_params(pm):
    R = np.arange(9.0).reshape(3, 3) / 7
    p = pm.make_pose((R, [1.5, -2.0, 0.25]))
    assert list(p.R) == list(R.reshape(9)) and list(p.t) == [1.5, -2.0, 0.25]
    d = pm.pmsp_default_params()
    q = pm.make_params(dict(patch_w=7, seed=9))
    for name, _ in pm.pmsp_params._fields_:
        want = {"patch_w": 7, "seed": 9}.get(name, getattr(d, name))
        assert getattr(q, name) == pytest.approx(want), name
    assert pm.make_params(q) is q
    with pytest.raises(KeyError):
        pm.make_params(dict(no_such_field=1))


def test_host_maps_and_batch(pm):
    m = pm.Maps.empty(12, 6)
    c = m.c()
    assert (c.w, c.h, c.memory) == (12, 6, pm.PMSP_HOST)
    assert (c.depth, c.normal, c.cost) == (m.depth.ctypes.data, m.normal.ctypes.data, m.cost.ctypes.data)
    assert m.normal.shape == (3, 6, 12)
    ref = np.zeros((6, 12), np.uint8)
    srcs = [np.full((6, 12), k, np.uint8) for k in range(3)]
    poses = [(np.eye(3), [0.1 * k, 0, 0]) for k in range(3)]
    b = pm.Batch([(ref, (np.eye(3), np.zeros(3)), srcs, poses, dict(best_k=2), None),
                  (ref, (np.eye(3), np.zeros(3)), srcs[:2], poses[:2], dict(best_k=1), None)])
    assert len(b) == 2 and [it.n_src for it in b.items] == [3, 2]
    assert [it.params.best_k for it in b.items] == [2, 1]
    assert b.items[0].srcs[2].data == srcs[2].ctypes.data and b.items[0].src_poses[1].t[0] == pytest.approx(0.1)
    assert b.items[1].out.w == 12 and b.items[1].out.memory == pm.PMSP_HOST
    with pytest.raises(ValueError):
        pm.Batch([(ref, (np.eye(3), np.zeros(3)), [], [], None, None)])
