"""CPU oracle (FP64) for PatchMatch-Stereo-Panorama densification.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library. It is a plain C
restatement of the method (oracle.c) with a ctypes wrapper, and it shares no
code with the CUDA path. Parity of every function here is pinned by
tests/test_oracle_*.py against closed forms, brute force and invariants.

Images enter as numpy arrays: uint8 (taken as DN/255), float16 or float32/64
(taken as given, expected in [0, 1]). Poses are world->camera (R 3x3, t 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
# PMSP_ORACLE_LIB names a prebuilt library to load instead of liboracle.so: the
# planted-mistake tests point it at builds of oracle.c with one mistake planted.
_PLANTED = os.environ.get("PMSP_ORACLE_LIB")
_LIB = _PLANTED or os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None
MAX_SRC = 16


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, OpenMP)."""
    if _PLANTED:
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Pose(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


class Params(ctypes.Structure):
    _fields_ = [("d_min", ctypes.c_double), ("d_max", ctypes.c_double),
                ("patch_w", ctypes.c_int32), ("patch_stride", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("best_k", ctypes.c_int32),
                ("sigma_color", ctypes.c_double), ("sigma_space", ctypes.c_double),
                ("n_refine", ctypes.c_int32), ("neighbor_table", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("keyframe_id", ctypes.c_uint64)]


class Img(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("I", ctypes.POINTER(ctypes.c_double))]


class ProblemC(ctypes.Structure):
    _fields_ = [("ref", Img), ("S", ctypes.c_int32), ("src", Img * MAX_SRC),
                ("rel", Pose * MAX_SRC), ("p", Params)]


_dp = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(ProblemC)
            lib.orc_bearing.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
            lib.orc_project.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            lib.orc_sample.argtypes = [ctypes.POINTER(Img), ctypes.c_double, ctypes.c_double]
            lib.orc_sample.restype = ctypes.c_double
            lib.orc_rel_pose.argtypes = [ctypes.POINTER(Pose)] * 3
            lib.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
            lib.orc_u24.argtypes = [ctypes.c_uint64]
            lib.orc_u24.restype = ctypes.c_double
            lib.orc_cost.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]
            lib.orc_cost.restype = ctypes.c_double
            lib.orc_cost_map.argtypes = [P, _dp, _dp, _dp]
            lib.orc_random_plane.argtypes = [P, ctypes.c_int, ctypes.c_int, _dp, _dp]
            lib.orc_init.argtypes = [P, _dp, _dp, _dp]
            lib.orc_neighbor_table.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.orc_neighbor_table.restype = ctypes.c_int
            lib.orc_update_pixel.argtypes = [P, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             _dp, _dp, _dp]
            lib.orc_halfsweep.argtypes = [P, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int]
            lib.orc_densify.argtypes = [P, _dp, _dp, _dp]
            lib.orc_plane_sweep.argtypes = [P, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
            lib.orc_warp_init.argtypes = [P, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.POINTER(Pose), _dp, _dp,
                                          _dp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            lib.orc_fuse.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(_dp), ctypes.POINTER(Pose), ctypes.c_double, _dp,
                                     ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, _dp]
            lib.orc_fuse.restype = ctypes.c_int64
            lib.orc_completeness.argtypes = [_dp, ctypes.c_int64, ctypes.POINTER(Pose), ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int), _dp]
            lib.orc_completeness.restype = ctypes.c_double
            lib.orc_view_filter.argtypes = [ctypes.POINTER(Pose), ctypes.POINTER(Pose), _dp, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp,
                                            ctypes.POINTER(ctypes.c_int), _dp]
            lib.orc_view_filter.restype = ctypes.c_int
            lib.orc_median_filter.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double,
                                              _dp, _dp]
            lib.orc_consistency_filter.argtypes = [
                ctypes.c_int, ctypes.c_int, _dp, ctypes.POINTER(Pose), ctypes.c_int,
                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_dp),
                ctypes.POINTER(Pose), ctypes.c_double, ctypes.c_int, _dp,
                ctypes.POINTER(ctypes.c_int), _dp]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def to_intensity(img) -> np.ndarray:
    """Image array -> float64 intensities (uint8 is DN/255)."""
    img = np.asarray(img)
    if img.dtype == np.uint8:
        return np.ascontiguousarray(img, dtype=np.float64) / 255.0
    return np.ascontiguousarray(img, dtype=np.float64)


def make_pose(R, t) -> Pose:
    p = Pose()
    R = np.asarray(R, dtype=np.float64).reshape(9)
    t = np.asarray(t, dtype=np.float64).reshape(3)
    for i in range(9):
        p.R[i] = float(R[i])
    for i in range(3):
        p.t[i] = float(t[i])
    return p


def rel_pose(R_r, t_r, R_s, t_s):
    """Reference->source pose (FP64): R = R_s R_r^T, t = t_s - R t_r."""
    lib = _load()
    out = Pose()
    a, b = make_pose(R_r, t_r), make_pose(R_s, t_s)
    lib.orc_rel_pose(ctypes.byref(a), ctypes.byref(b), ctypes.byref(out))
    return np.array(out.R[:]).reshape(3, 3), np.array(out.t[:])


DEFAULT_PARAMS = dict(d_min=0.3, d_max=10.0, patch_w=7, patch_stride=1, iterations=4, best_k=1,
                      sigma_color=0.0, sigma_space=0.0, n_refine=6, neighbor_table=0,
                      seed=42, keyframe_id=0)


class Problem:
    """A reference image, S source images with poses, and the parameters."""

    def __init__(self, ref_img, ref_pose, src_imgs, src_poses, **params):
        lib = _load()
        self._lib = lib
        self.ref = to_intensity(ref_img)
        self.srcs = [to_intensity(s) for s in src_imgs]
        if len(self.srcs) > MAX_SRC:
            raise ValueError("too many sources")
        self.H, self.W = self.ref.shape
        pr = dict(DEFAULT_PARAMS)
        pr.update(params)
        self.params = pr
        c = ProblemC()
        c.ref = Img(self.W, self.H, _ptr(self.ref))
        c.S = len(self.srcs)
        Rr, tr = ref_pose
        for s, (img, (Rs, ts)) in enumerate(zip(self.srcs, src_poses)):
            c.src[s] = Img(img.shape[1], img.shape[0], _ptr(img))
            lib.orc_rel_pose(ctypes.byref(make_pose(Rr, tr)), ctypes.byref(make_pose(Rs, ts)),
                             ctypes.byref(c.rel[s]))
        p = c.p
        for k in ("d_min", "d_max", "sigma_color", "sigma_space"):
            setattr(p, k, float(pr[k]))
        for k in ("patch_w", "patch_stride", "iterations", "best_k", "n_refine", "neighbor_table",
                  "seed", "keyframe_id"):
            setattr(p, k, int(pr[k]))
        self.c = c

    @classmethod
    def from_scene(cls, prob, **override):
        params = dict(prob.params)
        params.update(override)
        return cls(prob.ref.image, (prob.ref.R, prob.ref.t), [f.image for f in prob.srcs],
                   [(f.R, f.t) for f in prob.srcs], **params)

    # -- maps ---------------------------------------------------------------
    def _maps(self):
        N = self.W * self.H
        return (np.zeros((self.H, self.W)), np.zeros((3, self.H, self.W)), np.zeros((self.H, self.W)))

    def cost(self, u, v, d, n, per_view=False):
        n = np.ascontiguousarray(n, dtype=np.float64)
        vc = np.zeros(MAX_SRC)
        c = self._lib.orc_cost(ctypes.byref(self.c), int(u), int(v), float(d), _ptr(n), _ptr(vc))
        return (c, vc[: self.c.S].copy()) if per_view else c

    def cost_map(self, depth, normal):
        depth = np.ascontiguousarray(depth, dtype=np.float64)
        normal = np.ascontiguousarray(normal, dtype=np.float64)
        out = np.zeros((self.H, self.W))
        self._lib.orc_cost_map(ctypes.byref(self.c), _ptr(depth), _ptr(normal), _ptr(out))
        return out

    def random_plane(self, u, v):
        d = np.zeros(1)
        n = np.zeros(3)
        self._lib.orc_random_plane(ctypes.byref(self.c), int(u), int(v), _ptr(d), _ptr(n))
        return d[0], n

    def init(self):
        d, n, c = self._maps()
        self._lib.orc_init(ctypes.byref(self.c), _ptr(d), _ptr(n), _ptr(c))
        return d, n, c

    def update_pixel(self, depth, normal, cost, u, v, it):
        depth = np.ascontiguousarray(depth, dtype=np.float64)
        normal = np.ascontiguousarray(normal, dtype=np.float64)
        cost = np.ascontiguousarray(cost, dtype=np.float64)
        d, n, c = np.zeros(1), np.zeros(3), np.zeros(1)
        self._lib.orc_update_pixel(ctypes.byref(self.c), _ptr(depth), _ptr(normal), _ptr(cost),
                                   int(u), int(v), int(it), _ptr(d), _ptr(n), _ptr(c))
        return d[0], n, c[0]

    def halfsweep(self, depth, normal, cost, colour, it):
        """In-place half-sweep on float64 C-contiguous maps."""
        for a in (depth, normal, cost):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        self._lib.orc_halfsweep(ctypes.byref(self.c), _ptr(depth), _ptr(normal), _ptr(cost),
                                int(colour), int(it))

    def densify(self):
        d, n, c = self._maps()
        self._lib.orc_densify(ctypes.byref(self.c), _ptr(d), _ptr(n), _ptr(c))
        return d, n, c

    def warp_init(self, prev_depth, prev_normal, prev_pose, ref_pose):
        """Initialisation from the previous keyframe's plane map (Sec. III-B).
        Returns depth, normal, cost, winning source index (-1: random) and the
        'clear' mask (decisions away from their thresholds)."""
        pd = np.ascontiguousarray(prev_depth, dtype=np.float64)
        pn = np.ascontiguousarray(prev_normal, dtype=np.float64)
        rel = Pose()
        self._lib.orc_rel_pose(ctypes.byref(make_pose(*prev_pose)), ctypes.byref(make_pose(*ref_pose)),
                               ctypes.byref(rel))
        d, n, c = self._maps()
        src = np.zeros((self.H, self.W), np.int32)
        clear = np.zeros((self.H, self.W), np.int32)
        ip = ctypes.POINTER(ctypes.c_int)
        self._lib.orc_warp_init(ctypes.byref(self.c), pd.shape[1], pd.shape[0], _ptr(pd), _ptr(pn),
                                ctypes.byref(rel), _ptr(d), _ptr(n), _ptr(c), src.ctypes.data_as(ip),
                                clear.ctypes.data_as(ip))
        return d, n, c, src, clear.astype(bool)

    def plane_sweep(self, n_levels, normals):
        normals = np.ascontiguousarray(normals, dtype=np.float64).reshape(-1, 3)
        bc, bd = np.zeros((self.H, self.W)), np.zeros((self.H, self.W))
        self._lib.orc_plane_sweep(ctypes.byref(self.c), int(n_levels), _ptr(normals), len(normals),
                                  _ptr(bc), _ptr(bd))
        return bc, bd


def bearing(W, H, u, v):
    lib = _load()
    r = np.zeros(3)
    lib.orc_bearing(W, H, float(u), float(v), _ptr(r))
    return r


def project(W, H, Y):
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    uc, vc = np.zeros(1), np.zeros(1)
    lib.orc_project(W, H, _ptr(Y), _ptr(uc), _ptr(vc))
    return uc[0], vc[0]


def sample(img, uc, vc):
    lib = _load()
    I = to_intensity(img)
    im = Img(I.shape[1], I.shape[0], _ptr(I))
    return lib.orc_sample(ctypes.byref(im), float(uc), float(vc))


def philox4x64_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(x) for x in key])
    o = (ctypes.c_uint64 * 4)()
    lib.orc_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def u24(word):
    return _load().orc_u24(ctypes.c_uint64(int(word)))


def neighbor_table(table_id):
    lib = _load()
    buf = (ctypes.c_int * 16)()
    n = lib.orc_neighbor_table(int(table_id), buf)
    return [(buf[2 * k], buf[2 * k + 1]) for k in range(n)]


def consistency_filter(depth, pose_r, nbr_depths, nbr_poses, max_px=1.0, min_views=2):
    """Returns (filtered depth, per-pixel agreeing-view count, decision margin)."""
    lib = _load()
    depth = np.ascontiguousarray(depth, dtype=np.float64)
    H, W = depth.shape
    n = len(nbr_depths)
    Ds = [np.ascontiguousarray(d, dtype=np.float64) for d in nbr_depths]
    Wj = (ctypes.c_int * max(1, n))(*[d.shape[1] for d in Ds])
    Hj = (ctypes.c_int * max(1, n))(*[d.shape[0] for d in Ds])
    Dp = (_dp * max(1, n))(*[_ptr(d) for d in Ds])
    Pj = (Pose * max(1, n))(*[make_pose(R, t) for (R, t) in nbr_poses])
    pr = make_pose(*pose_r)
    out = np.zeros_like(depth)
    agree = np.zeros((H, W), dtype=np.int32)
    margin = np.zeros((H, W))
    lib.orc_consistency_filter(W, H, _ptr(depth), ctypes.byref(pr), n, Wj, Hj, Dp, Pj,
                               float(max_px), int(min_views), _ptr(out),
                               agree.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(margin))
    return out, agree, margin


def median_filter(depth, radius=2, tau=0.05):
    """Median post-filter (Sec. III-C, item 2). Returns (filtered depth, window median)."""
    lib = _load()
    depth = np.ascontiguousarray(depth, dtype=np.float64)
    H, W = depth.shape
    if not 0 <= radius <= 16:
        raise ValueError("radius must be in [0, 16]")
    out = np.zeros_like(depth)
    med = np.zeros_like(depth)
    lib.orc_median_filter(W, H, _ptr(depth), int(radius), float(tau), _ptr(out), _ptr(med))
    return out, med


def view_filter(pose_a, pose_b, points, min_deg=6.0, max_deg=60.0, min_frac=0.2):
    """View Filter (Sec. III-A, Eq. 1). Returns (accept, share in range, theta in degrees, in-range flags)."""
    lib = _load()
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    n = pts.shape[0]
    theta = np.zeros(n)
    flags = np.zeros(n, np.int32)
    frac = ctypes.c_double(0.0)
    acc = lib.orc_view_filter(ctypes.byref(make_pose(*pose_a)), ctypes.byref(make_pose(*pose_b)), _ptr(pts), n,
                              float(min_deg), float(max_deg), float(min_frac), _ptr(theta),
                              flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(frac))
    return bool(acc), frac.value, theta, flags.astype(bool)


def fuse(depths, poses, voxel=0.02):
    """Point-cloud fusion (Sec. III). Returns (points (m, 3) in key order, sources k << 32 | pixel,
    per-input-pixel voxel-face margin, -1 where there is no point)."""
    lib = _load()
    Ds = [np.ascontiguousarray(d, dtype=np.float64) for d in depths]
    n = len(Ds)
    Ws = (ctypes.c_int * max(1, n))(*[d.shape[1] for d in Ds])
    Hs = (ctypes.c_int * max(1, n))(*[d.shape[0] for d in Ds])
    Dp = (_dp * max(1, n))(*[_ptr(d) for d in Ds])
    Ps = (Pose * max(1, n))(*[make_pose(R, t) for (R, t) in poses])
    total = sum(d.size for d in Ds)
    pts = np.zeros((max(1, total), 3))
    src = np.zeros(max(1, total), np.int64)
    margin = np.zeros(max(1, total))
    m = lib.orc_fuse(n, Ws, Hs, Dp, Ps, float(voxel), _ptr(pts), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     total, _ptr(margin))
    return pts[:m], src[:m], margin[:total]


def completeness(points, pose, W=720, H=360):
    """Keyframe completeness (Sec. IV). Returns (share of pixels hit, hit flags (H, W), per-point margin)."""
    lib = _load()
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    hit = np.zeros((H, W), np.int32)
    margin = np.zeros(max(1, len(pts)))
    c = lib.orc_completeness(_ptr(pts), len(pts), ctypes.byref(make_pose(*pose)), int(W), int(H),
                             hit.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(margin))
    return c, hit.astype(bool), margin[:len(pts)]
