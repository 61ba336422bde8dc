"""Seeded procedural clip generator: the only input source shared by the oracle and the CUDA path.

It renders a static Lambertian scene (textured planes, rectangles, oriented boxes) with a moving
pinhole camera and applies the workloads' noise model (multiplicative depth noise, additive image
noise, pose perturbation of the cameras handed to the method).  It contains no gather or filter
arithmetic.  The per-pixel work runs in ``synth.c`` (plain C, OpenMP); this module builds the scene
layouts and camera paths and marshals arrays.

Presets
  ``planes3``      3 textured planes, camera translating 0.02 units/frame with rotational jitter
                   (the 160x90x16 tiny workload)
  ``room``         6 planes + 4 boxes, hand-held spline path with N(0, 0.3 deg) jitter (HD/1080p)
  ``exact_const``  constant-albedo fronto-parallel planes separated in depth, exact geometry
  ``exact_shift``  one textured fronto-parallel plane; the camera moves exactly one pixel
                   footprint per frame, so every reprojection lands on a pixel centre
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libssvp_synth.so")
_lib = None

PLANE, RECT, BOX = 0, 1, 2


class _Object(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("textured", ctypes.c_int32),
        ("c", ctypes.c_double * 3),
        ("ax", ctypes.c_double * 9),
        ("half", ctypes.c_double * 3),
        ("albedo", ctypes.c_double * 3),
        ("tex_freq", ctypes.c_double),
        ("tex_seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile synth.c into libssvp_synth.so (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        lib.synth_render.argtypes = [ctypes.POINTER(_Object), ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, dp, dp, dp, fp, fp, dp, ctypes.POINTER(ctypes.c_int32)]
        lib.synth_render_thinlens.argtypes = [ctypes.POINTER(_Object), ctypes.c_int, dp, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, fp]
        lib.synth_add_noise.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.c_double, ctypes.c_double, fp, fp, fp, fp]
        lib.synth_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, dp]
        lib.synth_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_normal.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


# ------------------------------------------------------------------ small rotation helpers

def rodrigues(w) -> np.ndarray:
    """Rotation matrix exp([w]_x) of an axis-angle vector (radians)."""
    w = np.asarray(w, dtype=np.float64)
    th = float(np.linalg.norm(w))
    if th < 1e-300:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * (Kx @ Kx)


def rot_y(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def normals(seed: int, stream: int, frame: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_normals(seed, stream, frame, n, _ptr(out, ctypes.c_double))
    return out


def intrinsics(W: int, H: int, fx: float | None = None) -> np.ndarray:
    """Pinhole K with pixel centres at integers: cx=(W-1)/2, cy=(H-1)/2, fx=fy=0.75*W unless given."""
    f = 0.75 * W if fx is None else float(fx)
    return np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])


# ------------------------------------------------------------------ scene layouts

def _obj(kind, c, U=None, V=None, N=None, axes=None, half=(0, 0, 0), albedo=(1, 1, 1), textured=True,
         freq=2.0, tex_seed=0):
    o = _Object()
    o.kind = kind
    o.textured = 1 if textured else 0
    o.c[:] = [float(x) for x in c]
    ax = np.asarray(axes, dtype=np.float64) if axes is not None else np.stack([U, V, N]).astype(np.float64)
    o.ax[:] = [float(x) for x in ax.reshape(-1)]
    o.half[:] = [float(x) for x in half]
    o.albedo[:] = [float(x) for x in albedo]
    o.tex_freq = float(freq)
    o.tex_seed = int(tex_seed) & 0xFFFFFFFFFFFFFFFF
    return o


def _plane_z(z, textured=True, albedo=(1, 1, 1), freq=2.0, seed=0, rect=None, center_xy=(0, 0), rot=None):
    """Plane facing the camera (-z normal), optionally a rectangle rotated by `rot` (3x3)."""
    R = np.eye(3) if rot is None else rot
    U, V, N = R @ np.array([1.0, 0, 0]), R @ np.array([0, 1.0, 0]), R @ np.array([0, 0, -1.0])
    c = (center_xy[0], center_xy[1], z)
    if rect is None:
        return _obj(PLANE, c, U, V, N, albedo=albedo, textured=textured, freq=freq, tex_seed=seed)
    return _obj(RECT, c, U, V, N, half=(rect[0], rect[1], 0), albedo=albedo, textured=textured, freq=freq,
                tex_seed=seed)


LIGHT = np.array([0.3, -1.0, -0.4]) / np.linalg.norm([0.3, -1.0, -0.4])  # towards the light


def scene_planes3(seed: int):
    s = seed * 1000
    return [
        _plane_z(7.5, freq=2.0, seed=s + 1),
        _obj(PLANE, (0, 1.2, 0), U=np.array([1.0, 0, 0]), V=np.array([0, 0, 1.0]), N=np.array([0, -1.0, 0]),
             freq=2.5, tex_seed=s + 2),
        _plane_z(4.0, freq=3.0, seed=s + 3, rect=(1.0, 0.7), center_xy=(0.4, -0.1), rot=rot_y(np.radians(30))),
    ]


def scene_room(seed: int):
    rng = np.random.default_rng(10_000 + seed)
    s = seed * 1000
    objs = [
        _plane_z(12.0 + rng.uniform(-1, 1), freq=1.5, seed=s + 1),
        _obj(PLANE, (0, 1.5, 0), U=np.array([1.0, 0, 0]), V=np.array([0, 0, 1.0]), N=np.array([0, -1.0, 0]),
             freq=2.0, tex_seed=s + 2),
        _obj(PLANE, (0, -2.2, 0), U=np.array([1.0, 0, 0]), V=np.array([0, 0, 1.0]), N=np.array([0, 1.0, 0]),
             freq=1.5, tex_seed=s + 3),
        _obj(PLANE, (-4.5, 0, 0), U=np.array([0, 0, 1.0]), V=np.array([0, 1.0, 0]), N=np.array([1.0, 0, 0]),
             freq=2.0, tex_seed=s + 4),
        _obj(PLANE, (5.0, 0, 0), U=np.array([0, 0, 1.0]), V=np.array([0, 1.0, 0]), N=np.array([-1.0, 0, 0]),
             freq=2.0, tex_seed=s + 5),
        _plane_z(6.5, freq=3.0, seed=s + 6, rect=(1.0, 1.2), center_xy=(-1.8, 0.2), rot=rot_y(np.radians(40))),
    ]
    for b in range(4):
        half = rng.uniform(0.3, 0.8, size=3)
        cx, cz = rng.uniform(-2.5, 2.5), rng.uniform(3.0, 9.0)
        cy = 1.5 - half[1] if b % 2 == 0 else rng.uniform(-1.0, 0.5)
        axes = rot_y(rng.uniform(0, np.pi / 2)).T  # rows = box axes in world coordinates
        objs.append(_obj(BOX, (cx, cy, cz), axes=axes, half=half, albedo=rng.uniform(0.6, 1.0, 3),
                         freq=rng.uniform(2.0, 4.0), tex_seed=s + 10 + b))
    return objs


def scene_exact_const():
    return [
        _plane_z(9.0, textured=False, albedo=(0.2, 0.3, 0.7)),
        _plane_z(5.0, textured=False, albedo=(0.2, 0.8, 0.3), rect=(0.9, 0.6), center_xy=(0.6, 0.3)),
        _plane_z(3.0, textured=False, albedo=(0.8, 0.2, 0.2), rect=(0.4, 0.3), center_xy=(-0.4, -0.2)),
    ]


# ------------------------------------------------------------------ camera paths

def _catmull_rom(P, t):
    """Uniform Catmull-Rom through control points P (n, d) at parameter t in [0, n-1]."""
    n = len(P)
    i = int(np.clip(np.floor(t), 0, n - 2))
    u = t - i
    p0, p1, p2, p3 = P[max(i - 1, 0)], P[i], P[i + 1], P[min(i + 2, n - 1)]
    return 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u
                  + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)


def _w2c(Rc, C):
    """world->camera [R|t] from camera-to-world rotation Rc and centre C."""
    R = Rc.T
    return np.concatenate([R, (-R @ C)[:, None]], axis=1)


def path_translate(F, seed, step=0.02, jitter_deg=0.5, start=(-0.15, 0.0, 0.0)):
    out = np.empty((F, 3, 4))
    for f in range(F):
        C = np.array(start) + np.array([step * f, 0.0, 0.0])
        w = np.radians(jitter_deg) * normals(seed, 4, f, 3) if jitter_deg else np.zeros(3)
        out[f] = _w2c(rodrigues(w), C)
    return out


def path_handheld(F, seed, speed=0.02, jitter_deg=0.3):
    rng = np.random.default_rng(20_000 + seed)
    seg = 15
    n_ctrl = F // seg + 4
    amp = np.array([1.2, 0.25, 0.5])
    om = speed / amp[0]
    ph = rng.uniform(0, 2 * np.pi, 3)
    ctrl = np.stack([amp * np.sin(np.array([1.0, 0.7, 0.5]) * om * seg * (i - 1) + ph) for i in range(n_ctrl)])
    ctrl = ctrl - ctrl[1] + rng.normal(0, 0.05, size=ctrl.shape)
    yaw_ctrl = rng.normal(0, np.radians(3.0), size=n_ctrl)
    pitch_ctrl = rng.normal(0, np.radians(1.5), size=n_ctrl)
    out = np.empty((F, 3, 4))
    for f in range(F):
        t = 1.0 + f / seg
        C = _catmull_rom(ctrl, t)
        yaw = _catmull_rom(yaw_ctrl[:, None], t)[0] - 0.12 * C[0]
        pitch = _catmull_rom(pitch_ctrl[:, None], t)[0]
        Rs = rot_y(yaw) @ rodrigues([pitch, 0, 0])
        w = np.radians(jitter_deg) * normals(seed, 4, f, 3)
        out[f] = _w2c(Rs @ rodrigues(w), C)
    return out


def perturb_poses(w2c, seed, sigma):
    """Cameras handed to the method: centre + N(0, sigma) per axis, rotation exp(N(0, sigma) rad) applied
    on the camera-to-world side."""
    out = np.empty_like(w2c)
    for f in range(len(w2c)):
        R, t = w2c[f, :, :3], w2c[f, :, 3]
        Rc, C = R.T, -R.T @ t
        nz = normals(seed, 3, f, 6) * sigma
        out[f] = _w2c(rodrigues(nz[:3]) @ Rc, C + nz[3:])
    return out


# ------------------------------------------------------------------ clips

@dataclass
class Clip:
    """A rendered clip.  Arrays are C-contiguous.

    rgb (F,H,W,3) f32 noisy input colour, depth (F,H,W) f32 noisy camera-z depth,
    clean (F,H,W,3) f32 noise-free render, depth_true (F,H,W) f32,
    K (F,3,3) f64, w2c (F,3,4) f64 cameras handed to the method, w2c_true exact cameras.
    """
    W: int
    H: int
    F: int
    K: np.ndarray
    w2c: np.ndarray
    w2c_true: np.ndarray
    rgb: np.ndarray
    depth: np.ndarray
    clean: np.ndarray
    depth_true: np.ndarray
    world: np.ndarray | None = None
    objid: np.ndarray | None = None
    meta: dict = field(default_factory=dict)


PRESETS = {
    # name: (scene, path, sigma_depth, sigma_pose, sigma_img)
    "planes3": dict(sigma_depth=0.01, sigma_pose=0.002, sigma_img=0.03),
    "room": dict(sigma_depth=0.02, sigma_pose=0.002, sigma_img=0.05),
    "exact_const": dict(sigma_depth=0.0, sigma_pose=0.0, sigma_img=0.0),
    "exact_shift": dict(sigma_depth=0.0, sigma_pose=0.0, sigma_img=0.0),
}


def scene_and_path(preset: str, W: int, H: int, F: int, seed: int):
    K = np.repeat(intrinsics(W, H)[None], F, axis=0)
    if preset == "planes3":
        return scene_planes3(seed), path_translate(F, seed, step=0.02, jitter_deg=0.5), K
    if preset == "room":
        return scene_room(seed), path_handheld(F, seed), K
    if preset == "exact_const":
        return scene_exact_const(), path_translate(F, seed, step=0.02, jitter_deg=0.0, start=(-0.1, 0, 0)), K
    if preset == "exact_shift":
        # a fronto-parallel plane at Z = fx / 32: one pixel footprint is exactly 2^-5 units, and the
        # camera moves by exactly that much per frame
        # fx is a power of two so K^-1 of a pixel centre, the plane hits and the camera centres are all
        # exactly representable: the same scene point gives bit-identical colours in every frame
        fx = float(2.0 ** round(np.log2(0.75 * W)))
        K = np.repeat(intrinsics(W, H, fx)[None], F, axis=0)
        Z = fx / 32.0
        objs = [_plane_z(Z, freq=4.0, seed=seed * 1000 + 7)]
        return objs, path_translate(F, seed, step=1.0 / 32.0, jitter_deg=0.0, start=(0.0, 0.0, 0.0)), K
    raise ValueError(f"unknown preset {preset!r}")


def render(objs, K, w2c, W, H, with_world=False):
    lib = _load()
    F = len(K)
    arr = (_Object * len(objs))(*objs)
    K = np.ascontiguousarray(K, dtype=np.float64)
    R = np.ascontiguousarray(w2c[:, :, :3], dtype=np.float64)
    t = np.ascontiguousarray(w2c[:, :, 3], dtype=np.float64)
    rgb = np.empty((F, H, W, 3), np.float32)
    depth = np.empty((F, H, W), np.float32)
    world = np.empty((F, H, W, 3), np.float64) if with_world else None
    objid = np.empty((F, H, W), np.int32) if with_world else None
    light = np.ascontiguousarray(LIGHT)
    lib.synth_render(arr, len(objs), _ptr(light, ctypes.c_double), W, H, F, _ptr(K, ctypes.c_double),
                     _ptr(R, ctypes.c_double), _ptr(t, ctypes.c_double), _ptr(rgb, ctypes.c_float),
                     _ptr(depth, ctypes.c_float), _ptr(world, ctypes.c_double), _ptr(objid, ctypes.c_int32))
    return rgb, depth, world, objid


def render_thinlens(objs, K, w2c, W, H, aperture, z_focus, n_lens=256):
    lib = _load()
    F = len(K)
    arr = (_Object * len(objs))(*objs)
    K = np.ascontiguousarray(K, dtype=np.float64)
    R = np.ascontiguousarray(w2c[:, :, :3], dtype=np.float64)
    t = np.ascontiguousarray(w2c[:, :, 3], dtype=np.float64)
    rgb = np.empty((F, H, W, 3), np.float32)
    light = np.ascontiguousarray(LIGHT)
    lib.synth_render_thinlens(arr, len(objs), _ptr(light, ctypes.c_double), W, H, F, _ptr(K, ctypes.c_double),
                              _ptr(R, ctypes.c_double), _ptr(t, ctypes.c_double), float(aperture), float(z_focus),
                              int(n_lens), _ptr(rgb, ctypes.c_float))
    return rgb


def add_noise(rgb, depth, seed, sigma_img, sigma_depth, frame0=0):
    lib = _load()
    F, H, W = depth.shape
    rgb_o = np.empty_like(rgb)
    depth_o = np.empty_like(depth)
    lib.synth_add_noise(W, H, F, frame0, seed, float(sigma_img), float(sigma_depth), _ptr(rgb, ctypes.c_float),
                        _ptr(depth, ctypes.c_float), _ptr(rgb_o, ctypes.c_float), _ptr(depth_o, ctypes.c_float))
    return rgb_o, depth_o


def make_clip(preset: str, W: int, H: int, F: int, seed: int = 0, with_world: bool = False,
              sigma_depth=None, sigma_pose=None, sigma_img=None) -> Clip:
    """Render a clip of `preset` and apply its noise model (overridable per sigma)."""
    p = dict(PRESETS[preset])
    if sigma_depth is not None:
        p["sigma_depth"] = sigma_depth
    if sigma_pose is not None:
        p["sigma_pose"] = sigma_pose
    if sigma_img is not None:
        p["sigma_img"] = sigma_img
    objs, w2c_true, K = scene_and_path(preset, W, H, F, seed)
    clean, depth_true, world, objid = render(objs, K, w2c_true, W, H, with_world)
    if p["sigma_img"] or p["sigma_depth"]:
        rgb, depth = add_noise(clean, depth_true, seed, p["sigma_img"], p["sigma_depth"])
    else:
        rgb, depth = clean.copy(), depth_true.copy()
    w2c = perturb_poses(w2c_true, seed, p["sigma_pose"]) if p["sigma_pose"] else w2c_true.copy()
    return Clip(W, H, F, K, w2c, w2c_true, rgb, depth, clean, depth_true, world, objid,
                meta=dict(preset=preset, seed=seed, objects=objs, **p))


def object_box(obj, margin: float = 0.0, y_range=None):
    """World-space axis-aligned bounds (xmin, ymin, zmin, xmax, ymax, zmax) of a BOX object, grown by
    margin and optionally clipped to y_range (to keep a floor or ceiling the box rests on out)."""
    ax = np.array(obj.ax[:]).reshape(3, 3)
    half = np.array(obj.half[:])
    ext = np.abs(ax).T @ half + margin
    c = np.array(obj.c[:])
    lo, hi = c - ext, c + ext
    if y_range is not None:
        lo[1], hi[1] = max(lo[1], y_range[0]), min(hi[1], y_range[1])
    return tuple(lo) + tuple(hi)


def shake_blur(clip: Clip, frames, shake_deg: float = 0.5, n_sub: int = 6, seed: int = 0) -> Clip:
    """Motion blur from a sudden camera shake during the exposure of each listed frame: the clean
    image becomes the mean of n_sub renders whose camera rotates from the frame's pose to a random
    rotation of shake_deg degrees (the frame's pose, depth and clean reference stay those of the
    sharp start pose); the frame's image noise is then drawn again with the same key.  Returns a
    new Clip whose rgb holds the blurred, noisy frames."""
    objs = clip.meta["objects"]
    rgb = clip.rgb.copy()
    rng = np.random.default_rng(40_000 + seed)
    for f in frames:
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        subs = np.empty((n_sub, 3, 4))
        R0, t0 = clip.w2c_true[f, :, :3], clip.w2c_true[f, :, 3]
        C = -R0.T @ t0
        for i in range(n_sub):
            Rs = rodrigues(np.radians(shake_deg) * (i / max(n_sub - 1, 1)) * axis) @ R0
            subs[i] = _w2c(Rs.T, C)
        img, _, _, _ = render(objs, np.repeat(clip.K[f:f + 1], n_sub, axis=0), subs, clip.W, clip.H)
        blurred = img.mean(axis=0, dtype=np.float64).astype(np.float32)[None]
        sig = clip.meta.get("sigma_img", 0.0)
        if sig:
            blurred, _ = add_noise(blurred, clip.depth_true[f:f + 1], clip.meta["seed"], sig, 0.0, frame0=f)
        rgb[f] = blurred[0]
    return Clip(clip.W, clip.H, clip.F, clip.K, clip.w2c, clip.w2c_true, rgb, clip.depth, clip.clean,
                clip.depth_true, clip.world, clip.objid, meta=dict(clip.meta, blurred=list(frames), shake_deg=shake_deg))


# ------------------------------------------------------------------ workload recipes

WORKLOADS = {
    # name: (preset, W, H, F, half_window, k) - window T=None means "all frames"
    "tiny": dict(preset="planes3", W=160, H=90, F=16, T=None, k=5),
    "hd": dict(preset="room", W=1280, H=720, F=60, T=15, k=7),
    "fhd": dict(preset="room", W=1920, H=1080, F=68, T=30, k=7),
}
