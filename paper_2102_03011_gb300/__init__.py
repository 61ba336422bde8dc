"""Python binding of libssvp.so, the GB300 scene-space gather-and-filter library.

Argument marshalling only: every step of the path runs in the library's CUDA kernels.  The
functions carry the names of the C entry points declared in ``include/ssvp.h``; they accept
torch tensors (host or CUDA) or numpy arrays where the C call takes a pointer, and raise
``SsvpError`` when the C call returns a non-zero status.  There is no CPU fallback: importing
this package fails when ``libssvp.so`` has not been built (``_build.build()``).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libssvp.so")

SSVP_OK, SSVP_EINVAL, SSVP_ENOMEM, SSVP_ECUDA = 0, -1, -2, -3
SSVP_ENOCLIP, SSVP_ENOCAM, SSVP_ETIMEOUT, SSVP_EDEVICE = -4, -5, -6, -7
SSVP_MEM_HOST, SSVP_MEM_DEVICE = 0, 1
SSVP_COLOUR_F32, SSVP_COLOUR_F16 = 0, 1
SSVP_MODE_DENOISE, SSVP_MODE_APERTURE, SSVP_MODE_LEARNED, SSVP_MODE_MEAN = 0, 1, 2, 3
SSVP_MODE_DEBLUR, SSVP_MODE_SHUTTER, SSVP_MODE_INPAINT, SSVP_MODE_SEMI = 4, 5, 6, 7
SSVP_GATHER_WINDOW, SSVP_GATHER_FRUSTUM, SSVP_GATHER_WINDOW_TMA = 0, 1, 2
SSVP_MAX_CLIPS, SSVP_MAX_K, SSVP_MAX_HALF_WINDOW = 64, 31, 127
(SSVP_TRACE_GATHER, SSVP_TRACE_APERTURE, SSVP_TRACE_FRUSTUM, SSVP_TRACE_SUPERRES, SSVP_TRACE_EXTRACT, SSVP_TRACE_INFER,
 SSVP_TRACE_TRAIN, SSVP_TRACE_ADAM, SSVP_TRACE_BATCH, SSVP_TRACE_LOAD, SSVP_TRACE_MASK, SSVP_TRACE_KINDS) = range(12)


class SsvpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ssvp error {code}: {msg}")
        self.code = code


class ssvp_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("k", ctypes.c_int32), ("half_window", ctypes.c_int32),
                ("frame_begin", ctypes.c_int32), ("frame_end", ctypes.c_int32),
                ("crop_x", ctypes.c_int32), ("crop_y", ctypes.c_int32), ("crop_w", ctypes.c_int32),
                ("crop_h", ctypes.c_int32), ("radius", ctypes.c_float), ("sigma_rgb", ctypes.c_float),
                ("sigma_xyz", ctypes.c_float), ("sigma_f", ctypes.c_float), ("aperture", ctypes.c_float),
                ("focal_depth", ctypes.c_float), ("a0", ctypes.c_float), ("lens_samples", ctypes.c_int32),
                ("cap", ctypes.c_int32), ("max_samples", ctypes.c_int32), ("conf_threshold", ctypes.c_float),
                ("gather", ctypes.c_int32), ("frustum_l", ctypes.c_float), ("near_plane", ctypes.c_float),
                ("far_plane", ctypes.c_float), ("sigma_area", ctypes.c_float), ("test_skip_mma", ctypes.c_int32),
                ("membership_out", ctypes.c_void_p),
                ("pixel_stats_out", ctypes.c_void_p)]


class ssvp_plan_config(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_int32), ("frame_chunk", ctypes.c_int32)]


class ssvp_train_config(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch_pixels", ctypes.c_int32), ("lr", ctypes.c_float),
                ("bce_weight", ctypes.c_float), ("seed", ctypes.c_uint64), ("init", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2102_03011_gb300._build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    P = ctypes.POINTER(ssvp_params)
    sig = {
        "ssvp_params_default": (None, [P]),
        "ssvp_create": (i, [ctypes.POINTER(vp), i, vp]),
        "ssvp_destroy": (None, [vp]),
        "ssvp_last_error": (ctypes.c_char_p, [vp]),
        "ssvp_set_stream": (i, [vp, vp]),
        "ssvp_load_clip": (i, [vp, i, i, i, i, vp, vp, i, i]),
        "ssvp_unload_clip": (i, [vp, i]),
        "ssvp_append_frames": (i, [vp, i, i, vp, vp, i, vp, i, vp]),
        "ssvp_set_cameras": (i, [vp, i, vp, i, vp]),
        "ssvp_gather_filter": (i, [vp, P, ctypes.POINTER(ctypes.c_int), i]),
        "ssvp_read_output": (i, [vp, i, i, i, vp, i]),
        "ssvp_output_device_ptr": (i, [vp, i, ctypes.POINTER(vp)]),
        "ssvp_read_stats": (i, [vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong),
                                ctypes.POINTER(ctypes.c_double)]),
        "ssvp_clip_median_depth": (i, [vp, i, ctypes.POINTER(f)]),
        "ssvp_set_shutter": (i, [vp, ctypes.POINTER(f), i]),
        "ssvp_superres": (i, [vp, P, i, i, vp]),
        "ssvp_set_mask": (i, [vp, i, vp, i]),
        "ssvp_mask_from_box": (i, [vp, i, ctypes.POINTER(ctypes.c_double)]),
        "ssvp_read_mask": (i, [vp, i, vp]),
        "ssvp_frame_sharpness": (i, [vp, i, ctypes.POINTER(ctypes.c_double)]),
        "ssvp_sync": (i, [vp]),
        "ssvp_median_depth_noalloc": (i, [vp, ctypes.c_ulonglong, vp, vp]),
        "ssvp_autotune": (i, [vp, P, ctypes.POINTER(ctypes.c_int), i, ctypes.POINTER(ssvp_plan_config)]),
        "ssvp_plan_create": (i, [vp, P, ctypes.POINTER(ctypes.c_int), i, ctypes.POINTER(ssvp_plan_config),
                                 ctypes.POINTER(vp)]),
        "ssvp_plan_launch": (i, [vp]),
        "ssvp_plan_update": (i, [vp]),
        "ssvp_plan_get_config": (i, [vp, ctypes.POINTER(ssvp_plan_config), ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_int)]),
        "ssvp_plan_destroy": (None, [vp]),
        "ssvp_set_mlp": (i, [vp, vp, vp, vp, vp]),
        "ssvp_get_mlp": (i, [vp, vp, vp, vp, vp]),
        "ssvp_learned_samples": (i, [vp, P, i, vp, vp, vp, vp]),
        "ssvp_train": (i, [vp, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp), i,
                           ctypes.POINTER(ssvp_train_config), vp]),
        "ssvp_mlp_grad": (i, [vp, P, i, vp, i, vp, vp]),
        "ssvp_trace_enable": (i, [vp, i]),
        "ssvp_trace_read": (i, [vp, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
        "ssvp_trace_kind_name": (ctypes.c_char_p, [i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _ptr(x):
    """(address, on_device) of a torch tensor, numpy array or raw address."""
    if x is None:
        return None, False
    if isinstance(x, int):
        return x, False
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), bool(x.is_cuda)
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, False
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _check(ctx, rc):
    if rc != SSVP_OK:
        msg = lib.ssvp_last_error(ctx)
        raise SsvpError(rc, msg.decode() if msg else "")


def ssvp_params_default() -> ssvp_params:
    p = ssvp_params()
    lib.ssvp_params_default(ctypes.byref(p))
    return p


def ssvp_create(cuda_device: int = 0, cuda_stream=None):
    """Returns a context handle; cuda_stream is a torch.cuda.Stream, a raw cudaStream_t or None."""
    ctx = ctypes.c_void_p()
    s = cuda_stream.cuda_stream if hasattr(cuda_stream, "cuda_stream") else cuda_stream
    _check(None, lib.ssvp_create(ctypes.byref(ctx), int(cuda_device), s))
    return ctx


def ssvp_destroy(ctx) -> None:
    lib.ssvp_destroy(ctx)


def ssvp_last_error(ctx=None) -> str:
    m = lib.ssvp_last_error(ctx)
    return m.decode() if m else ""


def ssvp_set_stream(ctx, cuda_stream) -> None:
    s = cuda_stream.cuda_stream if hasattr(cuda_stream, "cuda_stream") else cuda_stream
    _check(ctx, lib.ssvp_set_stream(ctx, s))


def ssvp_load_clip(ctx, clip_id: int, W: int, H: int, F: int, rgb, depth, mem_kind: int | None = None,
                   colour_fmt: int = SSVP_COLOUR_F32) -> None:
    (pr, dr), (pd, dd) = _ptr(rgb), _ptr(depth)
    if mem_kind is None:
        if dr != dd:
            raise ValueError("rgb and depth must both be on the host or both on the device")
        mem_kind = SSVP_MEM_DEVICE if dr else SSVP_MEM_HOST
    _check(ctx, lib.ssvp_load_clip(ctx, clip_id, W, H, F, pr, pd, mem_kind, colour_fmt))


def ssvp_unload_clip(ctx, clip_id: int) -> None:
    _check(ctx, lib.ssvp_unload_clip(ctx, clip_id))


def ssvp_append_frames(ctx, clip_id: int, n: int, rgb, depth, K, per_frame_K: int, w2c, mem_kind: int | None = None) -> None:
    import numpy as np
    (pr, dr), (pd, dd) = _ptr(rgb), _ptr(depth)
    if mem_kind is None:
        if dr != dd:
            raise ValueError("rgb and depth must both be on the host or both on the device")
        mem_kind = SSVP_MEM_DEVICE if dr else SSVP_MEM_HOST
    K = np.ascontiguousarray(K, dtype=np.float64)
    w2c = np.ascontiguousarray(w2c, dtype=np.float64)
    _check(ctx, lib.ssvp_append_frames(ctx, clip_id, int(n), pr, pd, mem_kind, K.ctypes.data, int(per_frame_K),
                                       w2c.ctypes.data))


def ssvp_set_cameras(ctx, clip_id: int, K, per_frame_K: int, w2c) -> None:
    import numpy as np
    K = np.ascontiguousarray(K, dtype=np.float64)
    w2c = np.ascontiguousarray(w2c, dtype=np.float64)
    _check(ctx, lib.ssvp_set_cameras(ctx, clip_id, K.ctypes.data, int(per_frame_K), w2c.ctypes.data))


def ssvp_gather_filter(ctx, params: ssvp_params, clip_ids) -> None:
    ids = (ctypes.c_int * len(clip_ids))(*[int(c) for c in clip_ids])
    _check(ctx, lib.ssvp_gather_filter(ctx, ctypes.byref(params), ids, len(clip_ids)))


def ssvp_read_output(ctx, clip_id: int, frame_begin: int, frame_end: int, dst, mem_kind: int | None = None) -> None:
    p, dev = _ptr(dst)
    if mem_kind is None:
        mem_kind = SSVP_MEM_DEVICE if dev else SSVP_MEM_HOST
    _check(ctx, lib.ssvp_read_output(ctx, clip_id, frame_begin, frame_end, p, mem_kind))


def ssvp_output_device_ptr(ctx, clip_id: int) -> int:
    out = ctypes.c_void_p()
    _check(ctx, lib.ssvp_output_device_ptr(ctx, clip_id, ctypes.byref(out)))
    return int(out.value or 0)


def ssvp_read_stats(ctx):
    """-> (examined, accepted, sum_w) of the last gather call."""
    e, a, w = ctypes.c_ulonglong(), ctypes.c_ulonglong(), ctypes.c_double()
    _check(ctx, lib.ssvp_read_stats(ctx, ctypes.byref(e), ctypes.byref(a), ctypes.byref(w)))
    return int(e.value), int(a.value), float(w.value)


def ssvp_trace_enable(ctx, on: bool = True) -> None:
    _check(ctx, lib.ssvp_trace_enable(ctx, int(bool(on))))


def ssvp_trace_read(ctx) -> dict:
    """-> {kind name: (launches, summed device ms)} of the traced work since the last read."""
    n = SSVP_TRACE_KINDS
    kind, launches, ms = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_double * n)()
    got = ctypes.c_int()
    _check(ctx, lib.ssvp_trace_read(ctx, n, kind, launches, ms, ctypes.byref(got)))
    return {ssvp_trace_kind_name(kind[j]): (int(launches[j]), float(ms[j])) for j in range(got.value)}


def ssvp_trace_kind_name(kind: int) -> str:
    return lib.ssvp_trace_kind_name(kind).decode()


def ssvp_clip_median_depth(ctx, clip_id: int) -> float:
    m = ctypes.c_float()
    _check(ctx, lib.ssvp_clip_median_depth(ctx, clip_id, ctypes.byref(m)))
    return float(m.value)


def ssvp_superres(ctx, params: ssvp_params, clip_id: int, scale: int, out) -> None:
    """Super-resolution (Eq. 6-7) into `out`, a device tensor or pointer of
    n_frames x (H scale) x (W scale) x 3 floats."""
    p, dev = _ptr(out)
    if not dev and not isinstance(out, int):
        raise ValueError("ssvp_superres writes device memory: pass a CUDA tensor or a device pointer")
    _check(ctx, lib.ssvp_superres(ctx, ctypes.byref(params), clip_id, scale, p))


def ssvp_set_mask(ctx, clip_id: int, mask, mem_kind: int | None = None) -> None:
    """Inpainting mask (Eq. 8-9): F*H*W bytes, nonzero = remove (host array or CUDA tensor)."""
    p, dev = _ptr(mask)
    _check(ctx, lib.ssvp_set_mask(ctx, clip_id, p, (SSVP_MEM_DEVICE if dev else SSVP_MEM_HOST) if mem_kind is None
                                  else mem_kind))


def ssvp_mask_from_box(ctx, clip_id: int, box) -> None:
    """Mask every pixel whose world point lies in box = (xmin, ymin, zmin, xmax, ymax, zmax)."""
    import numpy as np
    b = np.ascontiguousarray(box, dtype=np.float64)
    if b.shape != (6,):
        raise ValueError("box needs 6 values")
    _check(ctx, lib.ssvp_mask_from_box(ctx, clip_id, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def ssvp_read_mask(ctx, clip_id: int, n_frames: int, H: int, W: int):
    import numpy as np
    out = np.zeros((n_frames, H, W), np.uint8)
    _check(ctx, lib.ssvp_read_mask(ctx, clip_id, out.ctypes.data))
    return out


def ssvp_set_shutter(ctx, xi, half_window: int) -> None:
    """Eq. 10 shutter function: xi[j] weighs samples from J = O - half_window + j."""
    import numpy as np
    a = np.ascontiguousarray(xi, dtype=np.float32)
    if a.size != 2 * half_window + 1:
        raise ValueError(f"xi needs {2 * half_window + 1} values, got {a.size}")
    _check(ctx, lib.ssvp_set_shutter(ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), half_window))


def ssvp_frame_sharpness(ctx, clip_id: int, n_frames: int):
    """Eq. 5's per-frame blurriness measure (sum of gradient magnitudes) -> float64 array."""
    import numpy as np
    out = np.zeros(n_frames, np.float64)
    _check(ctx, lib.ssvp_frame_sharpness(ctx, clip_id, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def ssvp_sync(ctx) -> None:
    _check(ctx, lib.ssvp_sync(ctx))


def _device_f32(x, name, need):
    """Address of a contiguous CUDA float32 tensor on the current device holding >= need values."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (device memory), not {type(x).__name__}")
    if x.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, not {x.dtype}")
    if x.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {x.device}, the current device is cuda:{torch.cuda.current_device()}")
    if x.numel() < need:
        raise ValueError(f"{name} holds {x.numel()} values, {need} are needed")
    return _ptr(x)[0]


def ssvp_median_depth_noalloc(depth_dev, n: int, median_dev, cuda_stream=None) -> None:
    """Median of a device array with the library's fixed scratch (no allocation); see ssvp.h.
    depth_dev and median_dev must be float32 CUDA tensors on the current device; n values of
    depth_dev are read (n <= depth_dev.numel())."""
    pm = _device_f32(median_dev, "median_dev", 1)
    pd = _device_f32(depth_dev, "depth_dev", 0)
    if int(n) > depth_dev.numel():
        raise ValueError(f"n={int(n)} exceeds depth_dev's {depth_dev.numel()} values")
    s = cuda_stream.cuda_stream if hasattr(cuda_stream, "cuda_stream") else cuda_stream
    _check(None, lib.ssvp_median_depth_noalloc(pd, int(n), pm, s))


def ssvp_autotune(ctx, params: ssvp_params, clip_ids) -> ssvp_plan_config:
    ids = (ctypes.c_int * len(clip_ids))(*[int(c) for c in clip_ids])
    best = ssvp_plan_config()
    _check(ctx, lib.ssvp_autotune(ctx, ctypes.byref(params), ids, len(clip_ids), ctypes.byref(best)))
    return best


class Plan:
    """Handle of an ssvp_plan together with its context (for error text)."""

    def __init__(self, handle, ctx):
        self.handle, self.ctx = handle, ctx


def ssvp_plan_create(ctx, params: ssvp_params, clip_ids, config: ssvp_plan_config | None = None) -> Plan:
    ids = (ctypes.c_int * len(clip_ids))(*[int(c) for c in clip_ids])
    out = ctypes.c_void_p()
    cfg = ctypes.byref(config) if config is not None else None
    _check(ctx, lib.ssvp_plan_create(ctx, ctypes.byref(params), ids, len(clip_ids), cfg, ctypes.byref(out)))
    return Plan(out, ctx)


def ssvp_plan_launch(plan: Plan) -> None:
    _check(plan.ctx, lib.ssvp_plan_launch(plan.handle))


def ssvp_plan_update(plan: Plan) -> None:
    _check(plan.ctx, lib.ssvp_plan_update(plan.handle))


def ssvp_plan_get_config(plan: Plan):
    """-> (ssvp_plan_config, n_items, grid)"""
    cfg, n, g = ssvp_plan_config(), ctypes.c_longlong(), ctypes.c_int()
    _check(plan.ctx, lib.ssvp_plan_get_config(plan.handle, ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(g)))
    return cfg, int(n.value), int(g.value)


def ssvp_plan_destroy(plan: Plan) -> None:
    lib.ssvp_plan_destroy(plan.handle)
    plan.handle = None


def _f32(a, shape):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape}, got {a.shape}")
    return a


def ssvp_set_mlp(ctx, W1, b1, W2, b2) -> None:
    arrs = [_f32(W1, (64, 16)), _f32(b1, (64,)), _f32(W2, (2, 64)), _f32(b2, (2,))]
    _check(ctx, lib.ssvp_set_mlp(ctx, *[a.ctypes.data for a in arrs]))


def ssvp_get_mlp(ctx):
    """-> (W1 (64, 16), b1 (64,), W2 (2, 64), b2 (2,)) float32"""
    import numpy as np
    out = [np.zeros((64, 16), np.float32), np.zeros(64, np.float32), np.zeros((2, 64), np.float32), np.zeros(2, np.float32)]
    _check(ctx, lib.ssvp_get_mlp(ctx, *[a.ctypes.data for a in out]))
    return tuple(out)


def ssvp_learned_samples(ctx, params: ssvp_params, clip_id: int, feat, col, nsamp, plain) -> None:
    _check(ctx, lib.ssvp_learned_samples(ctx, ctypes.byref(params), clip_id, _ptr(feat)[0], _ptr(col)[0],
                                         _ptr(nsamp)[0], _ptr(plain)[0]))


def ssvp_train(ctx, params: ssvp_params, clip_ids, clean, cfg: ssvp_train_config):
    """clean: device tensors (F, H, W, 3) float32, one per clip -> per-step losses (numpy)."""
    import numpy as np
    ids = (ctypes.c_int * len(clip_ids))(*[int(c) for c in clip_ids])
    ptrs = (ctypes.c_void_p * len(clean))(*[_ptr(c)[0] for c in clean])
    losses = np.zeros(max(cfg.steps, 1), np.float32)
    _check(ctx, lib.ssvp_train(ctx, ctypes.byref(params), ids, ptrs, len(clip_ids), ctypes.byref(cfg),
                               losses.ctypes.data))
    return losses[:cfg.steps]


def ssvp_mlp_grad(ctx, params: ssvp_params, clip_id: int, pixels, clean):
    """Flat gradient W1 | b1 | W2 | b2 and the loss (1219 floats) at the current weights."""
    import numpy as np
    px = np.ascontiguousarray(pixels, dtype=np.int32)
    g = np.zeros(1219, np.float32)
    _check(ctx, lib.ssvp_mlp_grad(ctx, ctypes.byref(params), clip_id, px.ctypes.data, len(px), _ptr(clean)[0],
                                  g.ctypes.data))
    return g
