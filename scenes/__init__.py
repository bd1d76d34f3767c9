"""Seeded synthetic equirectangular scenes: the shared input generator.

Both the CUDA path and the CPU oracle are fed from here. The module holds no
densification arithmetic: it builds a room, places objects, draws a camera
trajectory and ray-casts panoramas with a procedural texture plus the ground
truth range of every pixel (see render.c for the conventions).

The paper evaluates on a recorded flight through a hall (Sec. IV); that data
set is not available, so these scenes stand in for it at the paper's
online-mode resolution (1920x960, Sec. IV) and at the other sizes the
workloads use.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render.c")
_LIB = os.path.join(_HERE, "librender.so")
_lock = threading.Lock()
_lib = None

ROOM_LO = np.array([-2.0, -1.25, -1.5])   # x (4 m), y down (2.5 m), z (3 m)
ROOM_HI = np.array([2.0, 1.25, 1.5])


def build(force: bool = False) -> str:
    """Compile render.c into librender.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Obj(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("tex_seed", ctypes.c_int32),
                ("c", ctypes.c_double * 3), ("r", ctypes.c_double),
                ("gain", ctypes.c_double), ("bias", ctypes.c_double)]


class _Desc(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("tex_seed", ctypes.c_int32), ("freq", ctypes.c_double),
                ("gain", ctypes.c_double), ("bias", ctypes.c_double),
                ("n_obj", ctypes.c_int32), ("obj", ctypes.POINTER(_Obj))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.scene_render.argtypes = [ctypes.POINTER(_Desc), dp, dp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, dp, dp]
            lib.scene_ray_range.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, dp, dp, dp]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class SceneObject:
    kind: int            # 0 sphere, 1 axis-aligned box
    centre: np.ndarray
    radius: float        # sphere radius or box half-extent
    tex_seed: int
    gain: float
    bias: float


@dataclass
class Scene:
    seed: int
    objects: list = field(default_factory=list)
    freq: float = 3.0
    wall_gain: float = 0.75
    wall_bias: float = 0.12
    lo: np.ndarray = field(default_factory=lambda: ROOM_LO.copy())
    hi: np.ndarray = field(default_factory=lambda: ROOM_HI.copy())

    def _desc(self):
        objs = (_Obj * max(1, len(self.objects)))()
        for i, o in enumerate(self.objects):
            objs[i].kind = o.kind
            objs[i].tex_seed = o.tex_seed
            for a in range(3):
                objs[i].c[a] = float(o.centre[a])
            objs[i].r = o.radius
            objs[i].gain = o.gain
            objs[i].bias = o.bias
        d = _Desc()
        for a in range(3):
            d.lo[a] = float(self.lo[a])
            d.hi[a] = float(self.hi[a])
        d.tex_seed = self.seed & 0x7FFFFFFF
        d.freq = self.freq
        d.gain = self.wall_gain
        d.bias = self.wall_bias
        d.n_obj = len(self.objects)
        d.obj = objs
        return d, objs

    def render(self, R, t, W, H, ss=2, with_range=True):
        """Panorama (H, W) float64 in DN units (unquantised) and range (H, W) or None."""
        lib = _load()
        d, keep = self._desc()
        R = np.ascontiguousarray(R, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.float64)
        img = np.empty((H, W), np.float64)
        rng = np.empty((H, W), np.float64) if with_range else None
        lib.scene_render(ctypes.byref(d), _dp(R), _dp(t), W, H, ss, _dp(img),
                         _dp(rng) if rng is not None else None)
        del keep
        return img, rng

    def ray_range(self, origins, dirs):
        lib = _load()
        d, keep = self._desc()
        o = np.ascontiguousarray(origins, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        out = np.empty(len(o), np.float64)
        lib.scene_ray_range(ctypes.byref(d), len(o), _dp(o), _dp(v), _dp(out))
        del keep
        return out


def rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def pose_from_centre(R_cw, C):
    """world->camera (R, t) from a camera->world rotation and a camera centre."""
    R = np.asarray(R_cw).T.copy()
    return R, -R @ np.asarray(C, dtype=np.float64)


def trajectory(n, seed=2000, margin=0.4, mean_step=0.15, max_yaw_deg=10.0):
    """Smooth random walk inside the room: list of (R, t, centre).

    Steps ~ N(mean_step, 0.03) clipped to [0.08, 0.25] m, heading diffusing by
    0.35 rad per step, reflected at `margin` from the walls; yaw changes by at
    most `max_yaw_deg` between frames, pitch and roll stay within a few degrees.
    """
    rng = np.random.default_rng(seed)
    lo = ROOM_LO + margin
    hi = ROOM_HI - margin
    lo[1], hi[1] = -0.5, 0.5
    pos = rng.uniform(lo, hi)
    heading = rng.uniform(0, 2 * math.pi)
    yaw = rng.uniform(-math.pi, math.pi)
    out = []
    for k in range(n):
        if k > 0:
            heading += rng.normal(0.0, 0.35)
            step = float(np.clip(rng.normal(mean_step, 0.03), 0.08, 0.25))
            d = np.array([math.sin(heading), rng.normal(0.0, 0.1), math.cos(heading)])
            d /= np.linalg.norm(d)
            new = pos + step * d
            for a in range(3):
                if new[a] < lo[a] or new[a] > hi[a]:
                    d[a] = -d[a]
                    if a != 1:
                        heading = math.atan2(d[0], d[2])
            new = np.clip(pos + step * d, lo, hi)
            pos = new
            yaw += math.radians(rng.uniform(-max_yaw_deg, max_yaw_deg))
        pitch = math.radians(float(np.clip(rng.normal(0, 2.0), -5, 5)))
        roll = math.radians(float(np.clip(rng.normal(0, 2.0), -5, 5)))
        R_cw = rot_y(yaw) @ rot_x(pitch) @ rot_z(roll)
        R, t = pose_from_centre(R_cw, pos)
        out.append((R, t, pos.copy()))
    return out


def _obj_distance(kind, c, r, pts):
    if kind == 0:
        return np.maximum(np.linalg.norm(pts - c, axis=1) - r, 0.0)
    q = np.maximum(np.abs(pts - c) - r, 0.0)
    return np.linalg.norm(q, axis=1)


def place_objects(seed, cams, n=20, clearance=0.3):
    """n spheres/boxes with radius 0.2-1 m, none within `clearance` of a camera.

    A placement is retried up to 200 times; every 40 failures the radius
    shrinks by 20 % (not below 0.2 m); an object that still does not fit is
    dropped.
    """
    rng = np.random.default_rng(seed)
    cams = np.asarray(cams, dtype=np.float64).reshape(-1, 3)
    objs = []
    for i in range(n):
        kind = int(rng.integers(0, 2))
        r = float(rng.uniform(0.2, 1.0))
        gain = float(rng.uniform(0.55, 0.8))
        bias = float(rng.uniform(0.08, 0.2))
        for attempt in range(200):
            if attempt and attempt % 40 == 0:
                r = max(0.2, r * 0.8)
            c = rng.uniform(ROOM_LO, ROOM_HI)
            if np.all(_obj_distance(kind, c, r, cams) > clearance):
                objs.append(SceneObject(kind, c, r, int(seed * 131 + i * 17 + 5), gain, bias))
                break
    return objs


def quantise_u8(img_dn):
    return np.clip(np.rint(img_dn), 0, 255).astype(np.uint8)


@dataclass
class Frame:
    R: np.ndarray
    t: np.ndarray
    centre: np.ndarray
    image: np.ndarray        # u8 (H, W) or f16 (H, W) in [0, 1]
    range: np.ndarray | None  # ground-truth range (H, W) float64


@dataclass
class Problem:
    """One densification problem: reference frame, sources and parameters."""
    ref: Frame
    srcs: list
    params: dict
    scene: Scene


def config0(seed=1000, W=256, H=128):
    """256x128 room-only problem: 1 reference + 2 sources offset 0.1-0.3 m."""
    rng = np.random.default_rng(seed)
    scene = Scene(seed=seed)
    lo, hi = ROOM_LO + 0.7, ROOM_HI - 0.7
    C = rng.uniform(lo, hi)
    yaw = rng.uniform(-math.pi, math.pi)
    R0, t0 = pose_from_centre(rot_y(yaw), C)
    img, rg = scene.render(R0, t0, W, H)
    ref = Frame(R0, t0, C, quantise_u8(img), rg)
    srcs = []
    for k in range(2):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Cs = C + rng.uniform(0.1, 0.3) * d
        Rs, ts = pose_from_centre(rot_y(yaw + math.radians(rng.uniform(-5, 5))), Cs)
        im, r = scene.render(Rs, ts, W, H)
        srcs.append(Frame(Rs, ts, Cs, quantise_u8(im), r))
    params = dict(d_min=0.3, d_max=10.0, patch_w=7, patch_stride=1, iterations=4, best_k=1,
                  sigma_color=0.0, sigma_space=0.0, n_refine=6, neighbor_table=0,
                  seed=42, keyframe_id=0)
    return Problem(ref, srcs, params, scene)


def trajectory_problem(W, H, n_src, seed_scene=1001, seed_traj=2000, n_objects=20,
                       noise_sigma=0.0, noise_seed=7, fmt="u8", offset=0, with_range=True):
    """Reference = middle frame of a (n_src + 1)-frame walk; sources = the others."""
    traj = trajectory(n_src + 1 + offset, seed=seed_traj)[offset:]
    scene = Scene(seed=seed_scene)
    scene.objects = place_objects(seed_scene + 77, [c for _, _, c in traj], n=n_objects)
    nrng = np.random.default_rng(noise_seed)
    frames = []
    for (R, t, C) in traj:
        img, rg = scene.render(R, t, W, H, with_range=with_range)
        if noise_sigma > 0:
            img = img + nrng.normal(0.0, noise_sigma, size=img.shape)
        im = quantise_u8(img) if fmt == "u8" else \
            (np.clip(img, 0, 255) / 255.0).astype(np.float16 if fmt == "f16" else np.float32)
        frames.append(Frame(R, t, C, im, rg))
    mid = n_src // 2
    ref = frames[mid]
    srcs = frames[:mid] + frames[mid + 1:]
    return Problem(ref, srcs, {}, scene)


def config1(W=1920, H=960, n_src=6, **kw):
    """1920x960, 6 sources, 11x11 window at stride 2, 8 iterations, best-3."""
    p = trajectory_problem(W, H, n_src, **kw)
    p.params = dict(d_min=0.3, d_max=10.0, patch_w=11, patch_stride=2, iterations=8, best_k=3,
                    sigma_color=0.2, sigma_space=3.0, n_refine=6, neighbor_table=0,
                    seed=42, keyframe_id=1)
    return p


def config2(W=3840, H=1920, n_src=8, fmt="f16", **kw):
    """3840x1920, 8 sources, 8-bit texture + N(0, 2 DN) noise, fp16 or u8 storage."""
    kw.setdefault("seed_scene", 1002)
    p = trajectory_problem(W, H, n_src, noise_sigma=2.0, fmt=fmt, **kw)
    p.params = dict(d_min=0.3, d_max=10.0, patch_w=11, patch_stride=2, iterations=8, best_k=3,
                    sigma_color=0.2, sigma_space=3.0, n_refine=6, neighbor_table=0,
                    seed=42, keyframe_id=2)
    return p
