"""FP64 CPU oracle of the scene-space gather-and-filter (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package.  It shares no code with the CUDA path (``paper_2102_03011_gb300``) and neither imports
the other; the only common dependency is the seeded input generator ``synth``.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over output pixels);
this module marshals arrays and holds the two steps that are plain library primitives:
the lower median of the valid input depths (a sort) and the derived default parameters.

Readings of the paper used here (Sec. "Denoising", Eq. 4; Sec. "Sample Gathering", Eq. 2):
  * depth is camera-space z; integer pixel coordinates are pixel centres;
  * the radius r defaults to 0.5 % of the clip's lower-median valid input depth;
  * colour is in [0, 1], so sigma_rgb = 40 / 255; sigma_f = 6 frames; sigma_xyz = r;
  * the k x k window is centred on floor(x + 0.5) of the projected reference point;
  * Eq. 5's blurriness is the sum over a frame of the forward-difference gradient magnitudes (L2
    over the colour channels and both axes, pixels with a right and a lower neighbour); Eq. 10's
    shutter function replaces the weight entirely;
  * the frustum gather (Eq. 1-2) takes Eq. 2's L1 distance as printed, strict, plus the frustum's
    own depth range (near, far) = (0.01, 1000) of Eq. 1, l = 3 pixels; it tests every pixel of
    every window frame.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libssvp_oracle.so")
_lib = None

MODE_DENOISE, MODE_APERTURE, MODE_MEAN, MODE_DEBLUR, MODE_SHUTTER = 0, 1, 3, 4, 5
GATHER_WINDOW, GATHER_FRUSTUM = 0, 1
CODE_OUT, CODE_INVALID, CODE_REJECT, CODE_ACCEPT, CODE_BAND = 0, 1, 2, 3, 8


class _Clip(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("F", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("rgb", ctypes.POINTER(ctypes.c_float)), ("depth", ctypes.POINTER(ctypes.c_float)),
                ("K", ctypes.POINTER(ctypes.c_double)), ("w2c", ctypes.POINTER(ctypes.c_double))]


class _Params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("k", ctypes.c_int32), ("T", ctypes.c_int32),
                ("lens_samples", ctypes.c_int32), ("radius", ctypes.c_double), ("sigma_rgb", ctypes.c_double),
                ("sigma_xyz", ctypes.c_double), ("sigma_f", ctypes.c_double), ("band_rel", ctypes.c_double),
                ("tie_band", ctypes.c_double), ("aperture", ctypes.c_double), ("focal_depth", ctypes.c_double),
                ("a0", ctypes.c_double), ("cap", ctypes.c_int32), ("gather", ctypes.c_int32),
                ("frustum_l", ctypes.c_double), ("near_plane", ctypes.c_double), ("far_plane", ctypes.c_double),
                ("frame_w", ctypes.POINTER(ctypes.c_double)), ("slot_w", ctypes.POINTER(ctypes.c_double)),
                ("sigma_area", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c into libssvp_oracle.so (gcc -O2, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp, fp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
        i32p, u8p, i64p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int64)
        lib.oc_compose.argtypes = [dp, dp, dp, dp, ctypes.c_int, dp, dp]
        lib.oc_weight_denoise.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oc_weight_denoise.restype = ctypes.c_double
        lib.oc_filter.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, dp]
        lib.oc_filter.restype = ctypes.c_double
        lib.oc_gather_filter.argtypes = [ctypes.POINTER(_Clip), ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, i64p, i64p, i32p, i32p,
                                         u8p, u8p, i32p]
        lib.oc_bruteforce.argtypes = [ctypes.POINTER(_Clip), ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, u8p]
        lib.oc_bruteforce.restype = ctypes.c_longlong
        lib.oc_frame_sharpness.argtypes = [ctypes.POINTER(_Clip), dp]
        lib.oc_mask_from_box.argtypes = [ctypes.POINTER(_Clip), dp, u8p]
        lib.oc_inpaint_filter.argtypes = [ctypes.POINTER(_Clip), ctypes.POINTER(_Params), u8p] + [ctypes.c_int] * 5 + \
            [dp, dp, i64p, i32p, ctypes.POINTER(ctypes.c_uint64), u8p]
        lib.oc_inpaint_filter.restype = ctypes.c_int
        lib.oc_semitransparent_filter.argtypes = lib.oc_inpaint_filter.argtypes
        lib.oc_semitransparent_filter.restype = ctypes.c_int
        lib.oc_weight_superres.argtypes = [dp, dp] + [ctypes.c_double] * 6
        lib.oc_weight_superres.restype = ctypes.c_double
        lib.oc_superres_filter.argtypes = [ctypes.POINTER(_Clip), ctypes.POINTER(_Params)] + [ctypes.c_int] * 6 + \
            [dp, dp, i64p, i32p, ctypes.POINTER(ctypes.c_uint64), u8p]
        lib.oc_frustum_filter.argtypes = [ctypes.POINTER(_Clip), ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, i64p, i32p,
                                          ctypes.POINTER(ctypes.c_uint64), u8p]
        lib.oc_learned_samples.argtypes = [ctypes.POINTER(_Clip), ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_int), dp]
        lib.oc_learned_samples.restype = ctypes.c_int
        lib.oc_learned_crop.argtypes = [ctypes.POINTER(_Clip), ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, i32p, dp]
        lib.oc_mlp_pixel.argtypes = [dp, dp, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, ctypes.c_double, dp, dp, dp,
                                     dp, dp]
        lib.oc_mlp_pixel.restype = ctypes.c_double
        lib.oc_mlp_loss_grad.argtypes = [ctypes.c_int, dp, dp, i32p, dp, dp, dp, dp, dp, dp, ctypes.c_int,
                                         ctypes.c_double, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.oc_mlp_loss_grad.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(t))


@dataclass
class Params:
    """Gather-and-filter parameters as the oracle reads them (absolute radius, absolute focal depth)."""
    mode: int = MODE_DENOISE
    k: int = 7
    T: int = 15
    radius: float = 0.025
    sigma_rgb: float = 40.0 / 255.0
    sigma_xyz: float | None = None      # None: equal to the radius
    sigma_f: float = 6.0
    band_rel: float = 1e-5
    tie_band: float = 1e-3
    aperture: float = 0.05
    focal_depth: float = 5.0
    a0: float | None = None             # None: half a pixel footprint at the focal depth (0.5 z0 / fx)
    lens_samples: int = 16
    cap: int = 31
    gather: int = GATHER_WINDOW
    frustum_l: float = 3.0              # Eq. 1-2: frustum size in pixels (the paper's usual l = 3)
    near_plane: float = 0.01            # Eq. 1: the paper's near and far depths
    far_plane: float = 1000.0
    frame_w: np.ndarray | None = None   # MODE_DEBLUR: Eq. 5's per-frame factor (F values), e.g. frame_sharpness()
    slot_w: np.ndarray | None = None    # MODE_SHUTTER: Eq. 10's xi(J - O) for J = O-T .. O+T (2T+1 values)
    sigma_area: float = 0.0             # super-resolution (Eq. 7) length scale; superres_filter fills 0 in

    def c_struct(self, fx: float) -> _Params:
        s = _Params()
        s.mode, s.k, s.T, s.lens_samples = self.mode, self.k, self.T, self.lens_samples
        s.radius = self.radius
        s.sigma_rgb, s.sigma_f = self.sigma_rgb, self.sigma_f
        s.sigma_xyz = self.radius if self.sigma_xyz is None else self.sigma_xyz
        s.band_rel, s.tie_band = self.band_rel, self.tie_band
        s.aperture, s.focal_depth = self.aperture, self.focal_depth
        s.a0 = 0.5 * self.focal_depth / fx if self.a0 is None else self.a0
        s.cap = self.cap
        s.gather = self.gather
        s.frustum_l, s.near_plane, s.far_plane = self.frustum_l, self.near_plane, self.far_plane
        keep = []
        for name in ("frame_w", "slot_w"):
            a = getattr(self, name)
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                setattr(s, name, _p(a, ctypes.c_double))
        s._keep = keep  # the arrays live as long as the struct
        s.sigma_area = self.sigma_area
        return s


class ClipView:
    """Keeps contiguous copies of a clip's arrays alive for the C side."""

    def __init__(self, rgb, depth, K, w2c):
        self.rgb = np.ascontiguousarray(rgb, dtype=np.float32)
        self.depth = np.ascontiguousarray(depth, dtype=np.float32)
        F, H, W = self.depth.shape
        self.K = np.ascontiguousarray(np.broadcast_to(K, (F, 3, 3)), dtype=np.float64)
        self.w2c = np.ascontiguousarray(w2c, dtype=np.float64)
        assert self.rgb.shape == (F, H, W, 3) and self.w2c.shape == (F, 3, 4)
        self.F, self.H, self.W = F, H, W
        s = _Clip()
        s.W, s.H, s.F = W, H, F
        s.rgb, s.depth = _p(self.rgb, ctypes.c_float), _p(self.depth, ctypes.c_float)
        s.K, s.w2c = _p(self.K, ctypes.c_double), _p(self.w2c, ctypes.c_double)
        self.c = s

    @classmethod
    def of(cls, clip):
        return cls(clip.rgb, clip.depth, clip.K, clip.w2c)


def median_depth(depth) -> float:
    """Lower median (rank floor((n-1)/2) of the sorted values) of the finite, positive depths."""
    d = np.asarray(depth, dtype=np.float32).reshape(-1)
    d = d[np.isfinite(d) & (d > 0)]
    if d.size == 0:
        raise ValueError("no valid depth")
    return float(np.sort(d)[(d.size - 1) // 2])


def default_params(clip_depth, mode=MODE_DENOISE, k=7, T=15, radius_rel=0.005, **kw) -> Params:
    r = radius_rel * median_depth(clip_depth)
    return Params(mode=mode, k=k, T=T, radius=r, **kw)


def compose(K_O, w2c_O, K_J, w2c_J, same: bool):
    """A1: returns (P_{J<-O}, G_{O<-J}) as 3x4 float64 arrays."""
    P, G = np.zeros((3, 4)), np.zeros((3, 4))
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (K_O, w2c_O, K_J, w2c_J)]
    _load().oc_compose(*[_p(a, ctypes.c_double) for a in args], int(same), _p(P, ctypes.c_double),
                       _p(G, ctypes.c_double))
    return P, G


def weight_denoise(s, sref, sigma_rgb, sigma_xyz, sigma_f) -> float:
    s = np.ascontiguousarray(s, dtype=np.float64)
    r = np.ascontiguousarray(sref, dtype=np.float64)
    return _load().oc_weight_denoise(_p(s, ctypes.c_double), _p(r, ctypes.c_double), sigma_rgb, sigma_xyz, sigma_f)


def filter_samples(S, sref, mode, sigma_rgb, sigma_xyz, sigma_f):
    """Eq. 3 over an explicit sample set S (n, 7) -> (colour (3,), W)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    r = np.ascontiguousarray(sref, dtype=np.float64)
    out = np.zeros(3)
    W = _load().oc_filter(_p(S, ctypes.c_double), len(S), _p(r, ctypes.c_double), mode, sigma_rgb, sigma_xyz,
                          sigma_f, _p(out, ctypes.c_double))
    return out, W


@dataclass
class Result:
    rgb: np.ndarray          # (ch, cw, 3) float64
    sumw: np.ndarray         # (ch, cw)
    nacc: np.ndarray         # (ch, cw) int64
    nexam: np.ndarray        # (ch, cw) int64
    status: np.ndarray | None = None   # (ch, cw, 2T+1) int32
    centre: np.ndarray | None = None   # (ch, cw, 2T+1, 2) int32
    amb: np.ndarray | None = None      # (ch, cw, 2T+1) uint8
    codes: np.ndarray | None = None    # (ch, cw, 2T+1, k, k) uint8 (aperture: cap x cap from the box origin)
    box: np.ndarray | None = None      # (ch, cw, 2T+1, 4) int32 (aperture)


def gather_filter(view: ClipView, prm: Params, O: int, crop=None, membership: bool = False) -> Result:
    """Run the oracle on output frame O over crop (x0, y0, w, h) (default: the full frame)."""
    x0, y0, cw, ch = crop if crop is not None else (0, 0, view.W, view.H)
    n, ns = cw * ch, 2 * prm.T + 1
    k = prm.cap if prm.mode == MODE_APERTURE else prm.k  # side of the per-slot code grid
    out = np.zeros((ch, cw, 3))
    sumw = np.zeros((ch, cw))
    nacc = np.zeros((ch, cw), np.int64)
    nexam = np.zeros((ch, cw), np.int64)
    st = ce = am = co = bx = None
    if membership:
        st = np.full((ch, cw, ns), -9, np.int32)
        ce = np.zeros((ch, cw, ns, 2), np.int32)
        am = np.zeros((ch, cw, ns), np.uint8)
        co = np.zeros((ch, cw, ns, k, k), np.uint8)
        bx = np.zeros((ch, cw, ns, 4), np.int32)
    ps = prm.c_struct(float(view.K[O, 0, 0]))
    rc = _load().oc_gather_filter(ctypes.byref(view.c), ctypes.byref(ps), O, x0, y0, cw, ch,
                                  _p(out, ctypes.c_double), _p(sumw, ctypes.c_double), _p(nacc, ctypes.c_int64),
                                  _p(nexam, ctypes.c_int64), _p(st, ctypes.c_int32), _p(ce, ctypes.c_int32),
                                  _p(am, ctypes.c_uint8), _p(co, ctypes.c_uint8), _p(bx, ctypes.c_int32))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return Result(out, sumw, nacc, nexam, st, ce, am, co, bx)


def bruteforce(view: ClipView, prm: Params, O: int, u: int, v: int, J: int) -> np.ndarray:
    """(H, W) uint8 map of every pixel of frame J within the radius of pixel (u, v) of frame O."""
    acc = np.zeros((view.H, view.W), np.uint8)
    ps = prm.c_struct(float(view.K[O, 0, 0]))
    _load().oc_bruteforce(ctypes.byref(view.c), ctypes.byref(ps), O, u, v, J, _p(acc, ctypes.c_uint8))
    return acc


@dataclass
class FrustumResult:
    rgb: np.ndarray          # (ch, cw, 3) float64
    sumw: np.ndarray         # (ch, cw)
    nacc: np.ndarray         # (ch, cw) int64
    count: np.ndarray | None = None  # (ch, cw, 2T+1) int32: samples per window frame
    hash: np.ndarray | None = None   # (ch, cw, 2T+1) uint64: sum of mix64(qy * W + qx + 1)
    band: np.ndarray | None = None   # (ch, cw, 2T+1) uint8: a tested pixel lies in the tie band


def frustum_filter(view: ClipView, prm: Params, O: int, crop=None, membership: bool = False) -> FrustumResult:
    """Frustum gather (Eq. 1-2) and the Eq. 3/4 filter on output frame O over crop (x0, y0, w, h)."""
    x0, y0, cw, ch = crop if crop is not None else (0, 0, view.W, view.H)
    ns = 2 * prm.T + 1
    out = np.zeros((ch, cw, 3))
    sumw = np.zeros((ch, cw))
    nacc = np.zeros((ch, cw), np.int64)
    cnt = hsh = bnd = None
    if membership:
        cnt = np.zeros((ch, cw, ns), np.int32)
        hsh = np.zeros((ch, cw, ns), np.uint64)
        bnd = np.zeros((ch, cw, ns), np.uint8)
    ps = prm.c_struct(float(view.K[O, 0, 0]))
    rc = _load().oc_frustum_filter(ctypes.byref(view.c), ctypes.byref(ps), O, x0, y0, cw, ch,
                                   _p(out, ctypes.c_double), _p(sumw, ctypes.c_double), _p(nacc, ctypes.c_int64),
                                   _p(cnt, ctypes.c_int32), _p(hsh, ctypes.c_uint64), _p(bnd, ctypes.c_uint8))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return FrustumResult(out, sumw, nacc, cnt, hsh, bnd)


def weight_superres(s, sref, dq, fxJ, sigma_rgb, sigma_xyz, sigma_f, sigma_area) -> float:
    """Eq. 7: Eq. 4 times exp(-s_area / (2 sigma_area^2)), s_area = (dq / fxJ)^2 (Eq. 6)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    r = np.ascontiguousarray(sref, dtype=np.float64)
    return _load().oc_weight_superres(_p(s, ctypes.c_double), _p(r, ctypes.c_double), float(dq), float(fxJ),
                                      sigma_rgb, sigma_xyz, sigma_f, sigma_area)


def superres_filter(view: ClipView, prm: Params, O: int, scale: int, crop=None, membership: bool = False,
                    sigma_area: float | None = None) -> FrustumResult:
    """Super-resolution (Eq. 6-7) of output frame O on the scale-times grid over an output-grid
    crop (x0, y0, w, h) (default: the whole grid).  sigma_area defaults to prm.sigma_area, else to
    one input-pixel footprint at the median depth (median depth / fx of O)."""
    Wh, Hh = view.W * scale, view.H * scale
    x0, y0, cw, ch = crop if crop is not None else (0, 0, Wh, Hh)
    ns = 2 * prm.T + 1
    out = np.zeros((ch, cw, 3))
    sumw = np.zeros((ch, cw))
    nacc = np.zeros((ch, cw), np.int64)
    cnt = hsh = bnd = None
    if membership:
        cnt = np.zeros((ch, cw, ns), np.int32)
        hsh = np.zeros((ch, cw, ns), np.uint64)
        bnd = np.zeros((ch, cw, ns), np.uint8)
    ps = prm.c_struct(float(view.K[O, 0, 0]))
    if sigma_area is not None:
        ps.sigma_area = sigma_area
    elif not prm.sigma_area > 0:
        ps.sigma_area = median_depth(view.depth) / float(view.K[O, 0, 0])
    rc = _load().oc_superres_filter(ctypes.byref(view.c), ctypes.byref(ps), O, scale, x0, y0, cw, ch,
                                    _p(out, ctypes.c_double), _p(sumw, ctypes.c_double), _p(nacc, ctypes.c_int64),
                                    _p(cnt, ctypes.c_int32), _p(hsh, ctypes.c_uint64), _p(bnd, ctypes.c_uint8))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return FrustumResult(out, sumw, nacc, cnt, hsh, bnd)


def mask_from_box(view: ClipView, box) -> np.ndarray:
    """Eq. 8-9's removal mask (F, H, W) uint8 from a world-space box (xmin, ymin, zmin, xmax, ymax, zmax)."""
    b = np.ascontiguousarray(box, dtype=np.float64)
    assert b.shape == (6,)
    m = np.zeros((view.F, view.H, view.W), np.uint8)
    _load().oc_mask_from_box(ctypes.byref(view.c), _p(b, ctypes.c_double), _p(m, ctypes.c_uint8))
    return m


def inpaint_filter(view: ClipView, prm: Params, mask, O: int, crop=None, membership: bool = False,
                   semi: bool = False) -> FrustumResult:
    """Inpainting (Eq. 8-9) of output frame O over crop (x0, y0, w, h) with the frustum gather;
    with semi, the semi-transparency variant (the pixel's own sample adds Eq. 4 weights to the
    second Eq. 9 step; prm.sigma_xyz and prm.sigma_f must be set)."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    assert mask.shape == (view.F, view.H, view.W)
    x0, y0, cw, ch = crop if crop is not None else (0, 0, view.W, view.H)
    ns = 2 * prm.T + 1
    out = np.zeros((ch, cw, 3))
    sumw = np.zeros((ch, cw))
    nacc = np.zeros((ch, cw), np.int64)
    cnt = hsh = bnd = None
    if membership:
        cnt = np.zeros((ch, cw, ns), np.int32)
        hsh = np.zeros((ch, cw, ns), np.uint64)
        bnd = np.zeros((ch, cw, ns), np.uint8)
    ps = prm.c_struct(float(view.K[O, 0, 0]))
    fn = _load().oc_semitransparent_filter if semi else _load().oc_inpaint_filter
    rc = fn(ctypes.byref(view.c), ctypes.byref(ps), _p(mask, ctypes.c_uint8), O, x0, y0, cw, ch,
            _p(out, ctypes.c_double), _p(sumw, ctypes.c_double), _p(nacc, ctypes.c_int64),
            _p(cnt, ctypes.c_int32), _p(hsh, ctypes.c_uint64), _p(bnd, ctypes.c_uint8))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return FrustumResult(out, sumw, nacc, cnt, hsh, bnd)


def frame_sharpness(view: ClipView) -> np.ndarray:
    """Eq. 5's blurriness measure per frame: the sum of forward-difference gradient magnitudes."""
    out = np.zeros(view.F)
    _load().oc_frame_sharpness(ctypes.byref(view.c), _p(out, ctypes.c_double))
    return out


def psnr(a, b) -> float:
    """10 log10(1 / MSE) over all values, peak 1, no clipping."""
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


# ------------------------------------------------------------------ learned per-sample weights

MAX_SAMPLES, N_FEAT, N_HID = 64, 16, 64


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def learned_crop(view: ClipView, prm: Params, O: int, crop=None):
    """Capped sample sets of a crop: features (ch, cw, 64, 16), colours (ch, cw, 64, 3), counts
    (ch, cw) and the plain Eq. 4 outputs (ch, cw, 3)."""
    x0, y0, cw, ch = crop if crop is not None else (0, 0, view.W, view.H)
    feat = np.zeros((ch, cw, MAX_SAMPLES, N_FEAT))
    col = np.zeros((ch, cw, MAX_SAMPLES, 3))
    n = np.zeros((ch, cw), np.int32)
    plain = np.zeros((ch, cw, 3))
    ps = prm.c_struct(float(view.K[O, 0, 0]))
    _load().oc_learned_crop(ctypes.byref(view.c), ctypes.byref(ps), O, x0, y0, cw, ch, _p(feat, ctypes.c_double),
                            _p(col, ctypes.c_double), _p(n, ctypes.c_int32), _p(plain, ctypes.c_double))
    return feat, col, n, plain


def mlp_pixel(feat, col, n, W1, b1, W2, b2, round_bf16=True, tau=0.5, plain=None):
    """Forward pass of one pixel -> (learned output, final output, conf, z (n, 2))."""
    feat, col = _d(feat).reshape(-1, N_FEAT), _d(col).reshape(-1, 3)
    W1, b1, W2, b2 = _d(W1), _d(b1), _d(W2), _d(b2)
    plain = _d(np.zeros(3) if plain is None else plain)
    ol, of, z = np.zeros(3), np.zeros(3), np.zeros((max(n, 1), 2))
    conf = _load().oc_mlp_pixel(_p(feat, ctypes.c_double), _p(col, ctypes.c_double), int(n), _p(W1, ctypes.c_double),
                                _p(b1, ctypes.c_double), _p(W2, ctypes.c_double), _p(b2, ctypes.c_double),
                                int(round_bf16), float(tau), _p(plain, ctypes.c_double), _p(ol, ctypes.c_double),
                                _p(of, ctypes.c_double), _p(z, ctypes.c_double), None)
    return ol, of, conf, z[:n]


def mlp_loss_grad(feat, col, nsamp, plain, clean, W1, b1, W2, b2, round_bf16=True, bce_w=0.1, term_scale=False):
    """Loss and gradients over pixels: feat (P, 64, 16), col (P, 64, 3), nsamp (P,), plain (P, 3),
    clean (P, 3) -> (L, gW1 (64, 16), gb1 (64,), gW2 (2, 64), gb2 (2,)).  With term_scale, also
    the per-entry sums of the absolute values of the terms (same shapes), appended."""
    feat, col, plain, clean = _d(feat), _d(col), _d(plain), _d(clean)
    nsamp = np.ascontiguousarray(nsamp, dtype=np.int32)
    W1, b1, W2, b2 = _d(W1), _d(b1), _d(W2), _d(b2)
    g = [np.zeros((N_HID, N_FEAT)), np.zeros(N_HID), np.zeros((2, N_HID)), np.zeros(2)]
    a = [np.zeros((N_HID, N_FEAT)), np.zeros(N_HID), np.zeros((2, N_HID)), np.zeros(2)] if term_scale else [None] * 4
    L = _load().oc_mlp_loss_grad(len(nsamp), _p(feat, ctypes.c_double), _p(col, ctypes.c_double),
                                 _p(nsamp, ctypes.c_int32), _p(plain, ctypes.c_double), _p(clean, ctypes.c_double),
                                 _p(W1, ctypes.c_double), _p(b1, ctypes.c_double), _p(W2, ctypes.c_double),
                                 _p(b2, ctypes.c_double), int(round_bf16), float(bce_w),
                                 *[_p(x, ctypes.c_double) for x in g], *[_p(x, ctypes.c_double) for x in a])
    return (L, *g, *a) if term_scale else (L, *g)


def he_init(seed=0):
    """He-normal W1 (64 x 16), W2 (2 x 64), zero biases (numpy RNG, seeded)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / 15), (N_HID, N_FEAT))  # 15 non-zero inputs
    W2 = rng.normal(0, np.sqrt(2.0 / N_HID), (2, N_HID))
    return W1, np.zeros(N_HID), W2, np.zeros(2)
