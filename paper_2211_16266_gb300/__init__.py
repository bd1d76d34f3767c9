"""Python binding of the GB300 PatchMatch-Stereo-Panorama densification library.

Argument marshalling only: every step of the densification runs in the CUDA
kernels of libpmsp.so behind the C ABI declared in include/pmsp.h. The
functions carry the C names (pmsp_create, pmsp_densify, ...). Arrays may be
numpy arrays (host memory) or torch tensors (device memory when on CUDA);
torch supplies device memory and streams only.

Importing this module fails loudly when libpmsp.so has not been built
(`python -c "import __graft_entry__ as g; g.build()"`); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PMSP_LIB") or os.path.join(_HERE, "libpmsp.so")  # PMSP_LIB: another build

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpmsp.so is missing at {LIB_PATH}: build the CUDA library first "
                      "(paper_2211_16266_gb300/_build.py); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

PMSP_OK = 0
PMSP_EINVAL = -1
PMSP_ENOMEM = -2
PMSP_EADMIT = -3
PMSP_EBUSY = -4
PMSP_ETIMEDOUT = -5
PMSP_ECUDA = -6
PMSP_EDEVICE = -7
PMSP_ENOTFOUND = -8
PMSP_U8, PMSP_F16, PMSP_F32 = 0, 1, 2
PMSP_HOST, PMSP_DEVICE = 0, 1
MAX_SOURCES = 16

_ERR_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "EADMIT", -4: "EBUSY", -5: "ETIMEDOUT",
              -6: "ECUDA", -7: "EDEVICE", -8: "ENOTFOUND"}


class PmspError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class pmsp_image(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("pitch_bytes", ctypes.c_int64),
                ("format", ctypes.c_int32), ("memory", ctypes.c_int32), ("data", ctypes.c_void_p)]


class pmsp_pose(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


class pmsp_params(ctypes.Structure):
    _fields_ = [("d_min", ctypes.c_float), ("d_max", ctypes.c_float), ("patch_w", ctypes.c_int32),
                ("patch_stride", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("best_k", ctypes.c_int32), ("sigma_color", ctypes.c_float),
                ("sigma_space", ctypes.c_float), ("n_refine", ctypes.c_int32),
                ("neighbor_table", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("keyframe_id", ctypes.c_uint64)]


class pmsp_maps(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("memory", ctypes.c_int32),
                ("depth", ctypes.c_void_p), ("normal", ctypes.c_void_p), ("cost", ctypes.c_void_p)]


class pmsp_ctx_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("stream", ctypes.c_void_p), ("mem_cap_bytes", ctypes.c_uint64),
                ("ring_capacity", ctypes.c_int32), ("max_active", ctypes.c_int32), ("scheduler", ctypes.c_int32)]


PMSP_SCHED_LANES, PMSP_SCHED_STEPS = 0, 1


_P = ctypes.c_void_p
_I = ctypes.POINTER(pmsp_image)
_O = ctypes.POINTER(pmsp_pose)
_R = ctypes.POINTER(pmsp_params)
_M = ctypes.POINTER(pmsp_maps)
_F = ctypes.c_void_p

_SIGS = {
    "pmsp_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(pmsp_ctx_opts)], ctypes.c_int),
    "pmsp_destroy": ([_P], ctypes.c_int),
    "pmsp_last_error": ([_P], ctypes.c_char_p),
    "pmsp_sync": ([_P], ctypes.c_int),
    "pmsp_default_params": ([_R], None),
    "pmsp_densify": ([_P, _I, _O, _I, _O, ctypes.c_int, _R, _M], ctypes.c_int),
    "pmsp_cost_map": ([_P, _I, _O, _I, _O, ctypes.c_int, _R, _M], ctypes.c_int),
    "pmsp_init": ([_P, _I, _O, _I, _O, ctypes.c_int, _R, _M], ctypes.c_int),
    "pmsp_halfsweep": ([_P, _I, _O, _I, _O, ctypes.c_int, _R, ctypes.c_int, ctypes.c_int, _M], ctypes.c_int),
    "pmsp_consistency_filter": ([_P, _M, _O, _M, _O, ctypes.c_int, ctypes.c_float, ctypes.c_int, _M, _F],
                                ctypes.c_int),
    "pmsp_sample_bilinear": ([_P, _I, ctypes.c_int, _F, _F, _F], ctypes.c_int),
    "pmsp_project": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _F, _F, _F, ctypes.c_int], ctypes.c_int),
}


class pmsp_batch_item(ctypes.Structure):
    _fields_ = [("ref", pmsp_image), ("ref_pose", pmsp_pose), ("srcs", ctypes.POINTER(pmsp_image)),
                ("src_poses", ctypes.POINTER(pmsp_pose)), ("n_src", ctypes.c_int32), ("params", pmsp_params),
                ("out", pmsp_maps)]


class pmsp_tuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("order", ctypes.c_int32), ("patch_stride", ctypes.c_int32),
                ("strategy", ctypes.c_int32), ("tile", ctypes.c_int32), ("tpp", ctypes.c_int32),
                ("lanes", ctypes.c_int32)]


class pmsp_peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_per_s", ctypes.c_double), ("fp32x2_fma_per_s", ctypes.c_double),
                ("sfu_per_s", ctypes.c_double), ("gather_l1_per_s", ctypes.c_double),
                ("gather_l2_per_s", ctypes.c_double), ("sm_clock_mhz_max", ctypes.c_double),
                ("sms", ctypes.c_int32), ("reserved", ctypes.c_int32)]


PMSP_BATCH_GRAPH = 1
_SIGS["pmsp_densify_batch"] = ([_P, ctypes.POINTER(pmsp_batch_item), ctypes.c_int, ctypes.c_uint32,
                                ctypes.POINTER(pmsp_tuning)], ctypes.c_int)
_SIGS["pmsp_autotune"] = ([_P, ctypes.POINTER(pmsp_batch_item), ctypes.c_int, ctypes.c_float,
                           ctypes.POINTER(pmsp_tuning)], ctypes.c_int)
_SIGS["pmsp_measure_peaks"] = ([_P, ctypes.POINTER(pmsp_peaks)], ctypes.c_int)
_SIGS["pmsp_densify_batch_noalloc"] = ([_P, ctypes.POINTER(pmsp_batch_item), ctypes.c_int], ctypes.c_int)
PMSP_NOALLOC_MAX_ITEMS = 16
_SIGS["pmsp_warp_init"] = ([_P, _I, _O, _I, _O, ctypes.c_int, _R, _M, _O, _M, _F], ctypes.c_int)
_SIGS["pmsp_densify_warped"] = ([_P, _I, _O, _I, _O, ctypes.c_int, _R, _M, _O, _M], ctypes.c_int)
_SIGS["pmsp_median_filter"] = ([_P, _M, ctypes.c_int, ctypes.c_float, _M], ctypes.c_int)
_SIGS["pmsp_view_filter"] = ([_P, _O, _O, _F, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, _F, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)],
                             ctypes.c_int)
_SIGS["pmsp_fuse"] = ([_P, _M, _O, ctypes.c_int, ctypes.c_float, _F, _F, ctypes.c_int64,
                       ctypes.POINTER(ctypes.c_int64)], ctypes.c_int)
_SIGS["pmsp_completeness"] = ([_P, _F, ctypes.c_int64, ctypes.c_int, _O, ctypes.c_int, ctypes.c_int, _F,
                               ctypes.POINTER(ctypes.c_double)], ctypes.c_int)
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

C_SYMBOLS = tuple(_SIGS)


# --------------------------------------------------------------- marshalling

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _format_of(dtype_name):
    return {"uint8": PMSP_U8, "float16": PMSP_F16, "float32": PMSP_F32}[dtype_name]


def make_image(arr, keep):
    """pmsp_image over a (H, W) numpy array or torch tensor (rows contiguous)."""
    if _is_torch(arr):
        if arr.dim() != 2 or arr.stride(1) != 1:
            raise ValueError("image must be a 2-D tensor with contiguous rows")
        fmt = _format_of(str(arr.dtype).replace("torch.", ""))
        im = pmsp_image(arr.shape[1], arr.shape[0], arr.stride(0) * arr.element_size(), fmt,
                        PMSP_DEVICE if arr.is_cuda else PMSP_HOST, arr.data_ptr())
    else:
        a = np.asarray(arr)
        if a.ndim != 2 or a.strides[1] != a.itemsize:
            a = np.ascontiguousarray(a)
        fmt = _format_of(a.dtype.name)
        im = pmsp_image(a.shape[1], a.shape[0], a.strides[0], fmt, PMSP_HOST, a.ctypes.data)
        arr = a
    keep.append(arr)
    return im


def make_pose(pose):
    R, t = pose
    p = pmsp_pose()
    R = np.asarray(R, dtype=np.float64).reshape(9)
    t = np.asarray(t, dtype=np.float64).reshape(3)
    for i in range(9):
        p.R[i] = float(R[i])
    for i in range(3):
        p.t[i] = float(t[i])
    return p


def pmsp_default_params(**override):
    p = pmsp_params()
    _lib.pmsp_default_params(ctypes.byref(p))
    for k, v in override.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def make_params(params):
    if isinstance(params, pmsp_params):
        return params
    return pmsp_default_params(**(params or {}))


class Maps:
    """Depth (H, W), normal (3, H, W) and cost (H, W) float32 buffers."""

    def __init__(self, depth, normal, cost):
        self.depth, self.normal, self.cost = depth, normal, cost

    @classmethod
    def empty(cls, W, H, device=None):
        if device is not None:
            import torch
            kw = dict(dtype=torch.float32, device=device)
            return cls(torch.empty((H, W), **kw), torch.empty((3, H, W), **kw), torch.empty((H, W), **kw))
        return cls(np.zeros((H, W), np.float32), np.zeros((3, H, W), np.float32), np.zeros((H, W), np.float32))

    def c(self):
        d = self.depth
        if _is_torch(d):
            for a in (self.depth, self.normal, self.cost):
                if a is not None:
                    assert a.is_contiguous() and str(a.dtype) == "torch.float32"
            mem = PMSP_DEVICE if d.is_cuda else PMSP_HOST
            ptr = lambda a: a.data_ptr() if a is not None else None
            H, W = d.shape
        else:
            for a in (self.depth, self.normal, self.cost):
                if a is not None:
                    assert a.dtype == np.float32 and a.flags.c_contiguous
            mem = PMSP_HOST
            ptr = lambda a: a.ctypes.data if a is not None else None
            H, W = d.shape
        return pmsp_maps(W, H, mem, ptr(self.depth), ptr(self.normal), ptr(self.cost))

    def numpy(self):
        f = (lambda a: a.detach().cpu().numpy()) if _is_torch(self.depth) else (lambda a: a)
        return f(self.depth), f(self.normal), f(self.cost)


def _ptr(a):
    if a is None:
        return None
    return a.data_ptr() if _is_torch(a) else a.ctypes.data


class Context:
    """Owns a pmsp_ctx. stream: "torch" (default: torch's current stream), a torch.cuda.Stream,
    a raw cudaStream_t int, or None (the context creates its own stream)."""

    def __init__(self, device=0, stream="torch", mem_cap_bytes=0, ring_capacity=0, max_active=0,
                 scheduler=PMSP_SCHED_LANES):
        # default: torch's current stream on `device`, so work is ordered after the
        # torch copies that produce the inputs; None: a private stream
        if isinstance(stream, str) and stream == "torch":
            import torch
            stream = torch.cuda.current_stream(device)
        raw = None
        if stream is not None:
            raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            if raw == 0:
                raw = 1  # torch's default stream is the legacy stream (cudaStreamLegacy)
        opts = pmsp_ctx_opts(device, raw, mem_cap_bytes, ring_capacity, max_active, scheduler)
        h = ctypes.c_void_p()
        rc = _lib.pmsp_create(ctypes.byref(h), ctypes.byref(opts))
        if rc != PMSP_OK:
            raise PmspError(rc, "pmsp_create failed")
        self.h = h

    def check(self, rc):
        if rc != PMSP_OK:
            raise PmspError(rc, _lib.pmsp_last_error(self.h).decode())
        return rc

    def close(self):
        if self.h:
            _lib.pmsp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def pmsp_create(device=0, stream="torch", **kw):
    return Context(device, stream, **kw)


def pmsp_destroy(ctx):
    ctx.close()


def pmsp_last_error(ctx):
    return _lib.pmsp_last_error(ctx.h).decode()


def pmsp_sync(ctx):
    return ctx.check(_lib.pmsp_sync(ctx.h))


def _problem(ref, ref_pose, srcs, src_poses, params, keep):
    n = len(srcs)
    if n < 1 or n > MAX_SOURCES or len(src_poses) != n:
        raise ValueError("need 1..16 sources with one pose each")
    cref = make_image(ref, keep)
    csrc = (pmsp_image * n)(*[make_image(s, keep) for s in srcs])
    cpose = (pmsp_pose * n)(*[make_pose(p) for p in src_poses])
    keep += [csrc, cpose]
    return cref, make_pose(ref_pose), csrc, cpose, n, make_params(params)


def _out_maps(ref, out):
    if out is not None:
        return out
    H, W = ref.shape
    return Maps.empty(W, H, device=ref.device if _is_torch(ref) and ref.is_cuda else None)


def pmsp_densify(ctx, ref, ref_pose, srcs, src_poses, params=None, out=None):
    """Densify one keyframe; returns Maps (device tensors for device input)."""
    keep = []
    cref, rp, cs, cp, n, p = _problem(ref, ref_pose, srcs, src_poses, params, keep)
    out = _out_maps(ref, out)
    m = out.c()
    ctx.check(_lib.pmsp_densify(ctx.h, ctypes.byref(cref), ctypes.byref(rp), cs, cp, n, ctypes.byref(p),
                                ctypes.byref(m)))
    return out


def pmsp_warp_init(ctx, ref, ref_pose, srcs, src_poses, params, prev, prev_pose, out=None, src=None):
    """Initialisation from the previous keyframe's maps (prev: Maps) by plane-map
    warping; returns the output Maps (device) and, if `src` is given, fills it."""
    keep = []
    cref, rp, cs, cp, n, p = _problem(ref, ref_pose, srcs, src_poses, params, keep)
    out = _out_maps(ref, out)
    pm_ = prev.c()
    m = out.c()
    ctx.check(_lib.pmsp_warp_init(ctx.h, ctypes.byref(cref), ctypes.byref(rp), cs, cp, n, ctypes.byref(p),
                                  ctypes.byref(pm_), ctypes.byref(make_pose(prev_pose)), ctypes.byref(m),
                                  _ptr(src)))
    return out


def pmsp_densify_warped(ctx, ref, ref_pose, srcs, src_poses, params, prev, prev_pose, out=None):
    """pmsp_densify starting from the previous keyframe's warped plane map."""
    keep = []
    cref, rp, cs, cp, n, p = _problem(ref, ref_pose, srcs, src_poses, params, keep)
    out = _out_maps(ref, out)
    pm_ = prev.c()
    m = out.c()
    ctx.check(_lib.pmsp_densify_warped(ctx.h, ctypes.byref(cref), ctypes.byref(rp), cs, cp, n, ctypes.byref(p),
                                       ctypes.byref(pm_), ctypes.byref(make_pose(prev_pose)), ctypes.byref(m)))
    return out


def pmsp_cost_map(ctx, ref, ref_pose, srcs, src_poses, params, planes):
    keep = []
    cref, rp, cs, cp, n, p = _problem(ref, ref_pose, srcs, src_poses, params, keep)
    m = planes.c()
    ctx.check(_lib.pmsp_cost_map(ctx.h, ctypes.byref(cref), ctypes.byref(rp), cs, cp, n, ctypes.byref(p),
                                 ctypes.byref(m)))
    return planes


def pmsp_init(ctx, ref, ref_pose, srcs, src_poses, params=None, out=None):
    keep = []
    cref, rp, cs, cp, n, p = _problem(ref, ref_pose, srcs, src_poses, params, keep)
    out = _out_maps(ref, out)
    m = out.c()
    ctx.check(_lib.pmsp_init(ctx.h, ctypes.byref(cref), ctypes.byref(rp), cs, cp, n, ctypes.byref(p),
                             ctypes.byref(m)))
    return out


def pmsp_halfsweep(ctx, ref, ref_pose, srcs, src_poses, params, colour, iteration, state):
    keep = []
    cref, rp, cs, cp, n, p = _problem(ref, ref_pose, srcs, src_poses, params, keep)
    m = state.c()
    ctx.check(_lib.pmsp_halfsweep(ctx.h, ctypes.byref(cref), ctypes.byref(rp), cs, cp, n, ctypes.byref(p),
                                  int(colour), int(iteration), ctypes.byref(m)))
    return state


def pmsp_consistency_filter(ctx, depth, pose, nbr_depths, nbr_poses, max_px=1.0, min_views=2, out=None,
                            agree=None):
    """Filter `depth` (H, W) against neighbour depth maps; returns (depth_out, agree)."""
    n = len(nbr_depths)
    if _is_torch(depth):
        import torch
        out = torch.empty_like(depth) if out is None else out
        if agree is None:
            agree = torch.empty(depth.shape, dtype=torch.int32, device=depth.device)
    else:
        depth = np.ascontiguousarray(depth, dtype=np.float32)
        nbr_depths = [np.ascontiguousarray(d, dtype=np.float32) for d in nbr_depths]
        out = np.zeros_like(depth) if out is None else out
        if agree is None:
            agree = np.zeros(depth.shape, np.int32)
    H, W = depth.shape
    mem = PMSP_DEVICE if _is_torch(depth) and depth.is_cuda else PMSP_HOST
    ref = pmsp_maps(W, H, mem, _ptr(depth), None, None)
    nb = (pmsp_maps * n)(*[pmsp_maps(d.shape[1], d.shape[0], mem, _ptr(d), None, None) for d in nbr_depths])
    poses = (pmsp_pose * n)(*[make_pose(p) for p in nbr_poses])
    o = pmsp_maps(W, H, mem, _ptr(out), None, None)
    ctx.check(_lib.pmsp_consistency_filter(ctx.h, ctypes.byref(ref), ctypes.byref(make_pose(pose)), nb, poses,
                                           n, float(max_px), int(min_views), ctypes.byref(o), _ptr(agree)))
    return out, agree


def pmsp_median_filter(ctx, depth, radius=2, tau=0.05, out=None):
    """Median post-filter of `depth` (H, W) (Sec. III-C, item 2); returns the filtered depth."""
    if _is_torch(depth):
        import torch
        out = torch.empty_like(depth) if out is None else out
    else:
        depth = np.ascontiguousarray(depth, dtype=np.float32)
        out = np.zeros_like(depth) if out is None else out
    H, W = depth.shape
    mem = PMSP_DEVICE if _is_torch(depth) and depth.is_cuda else PMSP_HOST
    src = pmsp_maps(W, H, mem, _ptr(depth), None, None)
    dst = pmsp_maps(W, H, mem, _ptr(out), None, None)
    ctx.check(_lib.pmsp_median_filter(ctx.h, ctypes.byref(src), int(radius), float(tau), ctypes.byref(dst)))
    return out


def _points(points):
    if _is_torch(points):
        return points, (PMSP_DEVICE if points.is_cuda else PMSP_HOST)
    return np.ascontiguousarray(np.asarray(points, dtype=np.float32).reshape(-1, 3)), PMSP_HOST


def pmsp_view_filter(ctx, pose_a, pose_b, points, min_deg=6.0, max_deg=60.0, min_frac=0.2, in_range=None):
    """View Filter (Sec. III-A, Eq. 1); returns (accepted, share in range, in-range flags or None)."""
    pts, mem = _points(points)
    n = int(pts.shape[0])
    acc = ctypes.c_int32(0)
    frac = ctypes.c_double(0.0)
    ctx.check(_lib.pmsp_view_filter(ctx.h, ctypes.byref(make_pose(pose_a)), ctypes.byref(make_pose(pose_b)),
                                    _ptr(pts), n, mem, float(min_deg), float(max_deg), float(min_frac),
                                    _ptr(in_range) if in_range is not None else None, ctypes.byref(acc),
                                    ctypes.byref(frac)))
    return bool(acc.value), frac.value, in_range


def pmsp_fuse(ctx, depths, poses, voxel=0.02, cap=None):
    """Point-cloud fusion (Sec. III); returns (points (m, 3), sources k << 32 | pixel, count)."""
    n = len(depths)
    dev = _is_torch(depths[0]) and depths[0].is_cuda
    mem = PMSP_DEVICE if dev else PMSP_HOST
    if not dev:
        depths = [np.ascontiguousarray(d, dtype=np.float32) for d in depths]
    maps = (pmsp_maps * n)(*[pmsp_maps(d.shape[1], d.shape[0], mem, _ptr(d), None, None) for d in depths])
    ps = (pmsp_pose * n)(*[make_pose(p) for p in poses])
    cnt = ctypes.c_int64(0)
    if cap is None:
        ctx.check(_lib.pmsp_fuse(ctx.h, maps, ps, n, float(voxel), None, None, 0, ctypes.byref(cnt)))
        cap = cnt.value
    if dev:
        import torch
        pts = torch.empty((max(1, cap), 3), dtype=torch.float32, device=depths[0].device)
        src = torch.empty(max(1, cap), dtype=torch.int64, device=depths[0].device)
    else:
        pts = np.zeros((max(1, cap), 3), np.float32)
        src = np.zeros(max(1, cap), np.int64)
    ctx.check(_lib.pmsp_fuse(ctx.h, maps, ps, n, float(voxel), _ptr(pts), _ptr(src), int(cap), ctypes.byref(cnt)))
    m = min(cnt.value, cap)
    return pts[:m], src[:m], cnt.value


def pmsp_completeness(ctx, points, pose, W=720, H=360, hit=None):
    """Keyframe completeness (Sec. IV); returns (share of pixels hit, hit flags or None)."""
    pts, mem = _points(points)
    out = ctypes.c_double(0.0)
    ctx.check(_lib.pmsp_completeness(ctx.h, _ptr(pts), int(pts.shape[0]), mem, ctypes.byref(make_pose(pose)),
                                     int(W), int(H), _ptr(hit) if hit is not None else None, ctypes.byref(out)))
    return out.value, hit


def pmsp_sample_bilinear(ctx, img, uc, vc):
    keep = []
    im = make_image(img, keep)
    if _is_torch(img):
        import torch
        out = torch.empty_like(uc)
    else:
        uc = np.ascontiguousarray(uc, dtype=np.float32)
        vc = np.ascontiguousarray(vc, dtype=np.float32)
        out = np.zeros_like(uc)
    ctx.check(_lib.pmsp_sample_bilinear(ctx.h, ctypes.byref(im), int(uc.shape[0]), _ptr(uc), _ptr(vc), _ptr(out)))
    return out


def pmsp_measure_peaks(ctx):
    """Measured FP32, special-function and gather rates of the device (dict)."""
    out = pmsp_peaks()
    ctx.check(_lib.pmsp_measure_peaks(ctx.h, ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in pmsp_peaks._fields_ if k != "reserved"}


def pmsp_project(ctx, W, H, dirs):
    """Continuous pixel coordinates (uc, vc) of (n, 3) directions in a W x H panorama."""
    if _is_torch(dirs):
        import torch
        d = dirs.contiguous()
        uc = torch.empty(d.shape[0], dtype=torch.float32, device=d.device)
        vc = torch.empty_like(uc)
        mem = PMSP_DEVICE if d.is_cuda else PMSP_HOST
    else:
        d = np.ascontiguousarray(dirs, dtype=np.float32).reshape(-1, 3)
        uc = np.zeros(d.shape[0], np.float32)
        vc = np.zeros_like(uc)
        mem = PMSP_HOST
    ctx.check(_lib.pmsp_project(ctx.h, int(W), int(H), int(d.shape[0]), _ptr(d), _ptr(uc), _ptr(vc), mem))
    return uc, vc


class Batch:
    """Marshalled pmsp_batch_item array; keeps every referenced buffer alive.

    problems: iterable of (ref, ref_pose, srcs, src_poses, params, out) where
    out is a Maps or None (allocated like pmsp_densify's output).
    """

    def __init__(self, problems):
        self.keep = []
        self.outs = []
        probs = list(problems)
        self.items = (pmsp_batch_item * len(probs))()
        for k, (ref, ref_pose, srcs, src_poses, params, out) in enumerate(probs):
            cref, rp, cs, cp, n, p = _problem(ref, ref_pose, srcs, src_poses, params, self.keep)
            out = _out_maps(ref, out)
            self.outs.append(out)
            it = self.items[k]
            it.ref, it.ref_pose, it.n_src, it.params, it.out = cref, rp, n, p, out.c()
            it.srcs = ctypes.cast(cs, ctypes.POINTER(pmsp_image))
            it.src_poses = ctypes.cast(cp, ctypes.POINTER(pmsp_pose))

    def __len__(self):
        return len(self.outs)


def pmsp_densify_batch(ctx, batch, flags=0, tuning=None):
    """Densify every problem of a Batch; returns the list of output Maps."""
    t = ctypes.byref(tuning) if tuning is not None else None
    ctx.check(_lib.pmsp_densify_batch(ctx.h, batch.items, len(batch), int(flags), t))
    return batch.outs


def pmsp_densify_batch_noalloc(ctx, batch):
    """pmsp_densify_batch without any device allocation (device-memory batches
    of at most PMSP_NOALLOC_MAX_ITEMS keyframes), for callers that must not
    allocate when they densify; see include/pmsp.h."""
    ctx.check(_lib.pmsp_densify_batch_noalloc(ctx.h, batch.items, len(batch)))
    return batch.outs


def pmsp_autotune(ctx, batch, max_changed=0.005):
    t = pmsp_tuning()
    ctx.check(_lib.pmsp_autotune(ctx.h, batch.items, len(batch), float(max_changed), ctypes.byref(t)))
    return t


# ------------------------------------------------------------------- serving

class pmsp_request(ctypes.Structure):
    _fields_ = [("ref_frame", ctypes.c_int64), ("n_src", ctypes.c_int32),
                ("src_frames", ctypes.POINTER(ctypes.c_int64)), ("params", pmsp_params),
                ("n_filter", ctypes.c_int32), ("filter_frames", ctypes.POINTER(ctypes.c_int64)),
                ("max_reproj_px", ctypes.c_float), ("min_views", ctypes.c_int32)]


class pmsp_serving_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("queued", ctypes.c_uint32), ("active", ctypes.c_uint32), ("steps", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64)]


for _name, _args in {
    "pmsp_ring_push": [_P, ctypes.c_int64, _I, _O],
    "pmsp_submit": [_P, ctypes.POINTER(pmsp_request), ctypes.POINTER(ctypes.c_uint64)],
    "pmsp_poll": [_P, ctypes.c_uint64, _M],
    "pmsp_wait": [_P, ctypes.c_uint64, ctypes.c_int, _M],
    "pmsp_get_serving_stats": [_P, ctypes.POINTER(pmsp_serving_stats)],
}.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int
C_SYMBOLS = C_SYMBOLS + ("pmsp_ring_push", "pmsp_submit", "pmsp_poll", "pmsp_wait", "pmsp_get_serving_stats")


def pmsp_ring_push(ctx, frame_id, image, pose):
    keep = []
    im = make_image(image, keep)
    ctx.check(_lib.pmsp_ring_push(ctx.h, int(frame_id), ctypes.byref(im), ctypes.byref(make_pose(pose))))


def pmsp_submit(ctx, ref_frame, src_frames, params=None, filter_frames=(), max_reproj_px=1.0, min_views=2):
    """Queue a densification request; returns its ticket."""
    srcs = (ctypes.c_int64 * len(src_frames))(*[int(f) for f in src_frames])
    filt = (ctypes.c_int64 * max(1, len(filter_frames)))(*[int(f) for f in filter_frames])
    req = pmsp_request(int(ref_frame), len(src_frames), srcs, make_params(params), len(filter_frames), filt,
                       float(max_reproj_px), int(min_views))
    t = ctypes.c_uint64()
    ctx.check(_lib.pmsp_submit(ctx.h, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def pmsp_poll(ctx, ticket, out=None):
    """Maps if finished (copied into `out`), None while queued or running."""
    m = out.c() if out is not None else None
    rc = _lib.pmsp_poll(ctx.h, int(ticket), ctypes.byref(m) if m is not None else None)
    if rc == PMSP_EBUSY:
        return None
    ctx.check(rc)
    return out


def pmsp_wait(ctx, ticket, timeout_ms, out=None):
    m = out.c() if out is not None else None
    ctx.check(_lib.pmsp_wait(ctx.h, int(ticket), int(timeout_ms), ctypes.byref(m) if m is not None else None))
    return out


def pmsp_get_serving_stats(ctx):
    s = pmsp_serving_stats()
    ctx.check(_lib.pmsp_get_serving_stats(ctx.h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_}
