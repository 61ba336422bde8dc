"""Pins of the oracle's per-frame weights: deblurring (Sec. "Deblurring", Eq. 5) and the
computational shutter (Sec. "Computational scene-space shutters", Eq. 10).

Closed forms used here:
  * the blurriness sum of a colour ramp I_c(x, y) = a_c x + b_c y is (W-1)(H-1) |(a, b)|, of a
    two-colour checkerboard (W-1)(H-1) sqrt(6) d for a grey step d; it ignores an added constant
    and scales with the image;
  * a frame with zero blurriness sum contributes to Eq. 5 exactly as if its depths were invalid;
  * equal per-frame factors (or a single frame) reduce Eq. 5 to Eq. 4;
  * a box shutter (xi = 1) is the plain average; on the one-pixel-per-frame translation scene with
    a colour offset per frame, a decaying shutter gives the xi-weighted mean of the offsets.
"""
import numpy as np
import pytest

import oracle
import synth


def _clip_with(rgb, depth=None, seed=0):
    F, H, W, _ = rgb.shape
    c = synth.make_clip("planes3", W, H, F, seed=seed)
    return oracle.ClipView(rgb, c.depth if depth is None else depth, c.K, c.w2c)


def test_sharpness_of_ramps_and_checkerboards():
    F, H, W = 3, 17, 29
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    rgb = np.zeros((F, H, W, 3), np.float32)
    ab = [((0.01, -0.02, 0.005), (0.0, 0.01, 0.02)), ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))]
    for f, (a, b) in enumerate(ab):
        for c in range(3):
            rgb[f, :, :, c] = 0.3 + a[c] * x + b[c] * y
    d = 0.25
    rgb[2] = (0.4 + d * ((x + y) % 2))[..., None]
    g = oracle.frame_sharpness(_clip_with(rgb))
    # float32 storage of the ramps: the differences are exact to ~1e-7 relative
    want0 = (W - 1) * (H - 1) * np.sqrt(sum(a * a + b * b for a, b in zip(*ab[0])))
    assert g[0] == pytest.approx(want0, rel=1e-5)
    assert g[1] == 0.0
    assert g[2] == pytest.approx((W - 1) * (H - 1) * np.sqrt(6.0) * d, rel=1e-6)
    g2 = oracle.frame_sharpness(_clip_with(rgb + np.float32(0.125)))
    np.testing.assert_allclose(g2, g, rtol=1e-5)
    g3 = oracle.frame_sharpness(_clip_with(rgb * np.float32(2.0)))
    np.testing.assert_allclose(g3, 2 * g, rtol=1e-6)


@pytest.fixture(scope="module")
def room():
    return synth.make_clip("room", 48, 27, 7, seed=6)


def test_zero_blurriness_frame_counts_as_absent(room):
    rgb = room.rgb.copy()
    rgb[5] = 0.5  # a frame with no gradient at all
    depth_holes = room.depth.copy()
    depth_holes[5] = np.nan
    v = oracle.ClipView(rgb, room.depth, room.K, room.w2c)
    g = oracle.frame_sharpness(v)
    assert g[5] == 0.0 and (np.delete(g, 5) > 0).all()
    p = oracle.default_params(room.depth, mode=oracle.MODE_DEBLUR, k=5, T=3, radius_rel=0.03, frame_w=g)
    a = oracle.gather_filter(v, p, 3)
    b = oracle.gather_filter(oracle.ClipView(rgb, depth_holes, room.K, room.w2c), p, 3)
    np.testing.assert_array_equal(a.rgb, b.rgb)
    assert (a.nacc >= b.nacc).all() and (a.nacc > b.nacc).any()  # the frame's samples are gathered, at weight 0
    # the same holds for the frustum gather
    for q in (p,):
        q.gather, q.sigma_xyz = oracle.GATHER_FRUSTUM, 0.03 * oracle.median_depth(room.depth)
        fa = oracle.frustum_filter(v, q, 3, crop=(10, 5, 12, 8))
        fb = oracle.frustum_filter(oracle.ClipView(rgb, depth_holes, room.K, room.w2c), q, 3, crop=(10, 5, 12, 8))
        np.testing.assert_array_equal(fa.rgb, fb.rgb)


def test_equal_factors_or_a_single_frame_reduce_to_eq4(room):
    v = oracle.ClipView.of(room)
    g = oracle.frame_sharpness(v)
    base = oracle.default_params(room.depth, k=5, T=3, radius_rel=0.03)
    den = oracle.gather_filter(v, base, 3)
    p = oracle.default_params(room.depth, mode=oracle.MODE_DEBLUR, k=5, T=3, radius_rel=0.03, frame_w=np.full(room.F, 7.0))
    np.testing.assert_allclose(oracle.gather_filter(v, p, 3).rgb, den.rgb, atol=1e-13, rtol=0)
    p1 = oracle.default_params(room.depth, mode=oracle.MODE_DEBLUR, k=5, T=0, radius_rel=0.03, frame_w=g)
    d1 = oracle.gather_filter(v, oracle.default_params(room.depth, k=5, T=0, radius_rel=0.03), 3)
    np.testing.assert_allclose(oracle.gather_filter(v, p1, 3).rgb, d1.rgb, atol=1e-13, rtol=0)
    # with the measured factors the result differs from Eq. 4 (the frames are not equally sharp)
    pg = oracle.default_params(room.depth, mode=oracle.MODE_DEBLUR, k=5, T=3, radius_rel=0.03, frame_w=g)
    assert np.abs(oracle.gather_filter(v, pg, 3).rgb - den.rgb).max() > 1e-6


def test_box_shutter_is_the_plain_average(room):
    v = oracle.ClipView.of(room)
    mean = oracle.gather_filter(v, oracle.default_params(room.depth, mode=oracle.MODE_MEAN, k=5, T=3, radius_rel=0.03), 3)
    box = oracle.default_params(room.depth, mode=oracle.MODE_SHUTTER, k=5, T=3, radius_rel=0.03, slot_w=np.ones(7))
    np.testing.assert_array_equal(oracle.gather_filter(v, box, 3).rgb, mean.rgb)


def test_decaying_shutter_closed_form_on_exact_shift():
    """Pixel (u, v) of O is seen at (u - (J - O), v) of J with the same colour c; adding an offset
    delta_J to all of frame J makes the shutter result c + sum xi delta / sum xi over the frames
    in which the point stays inside the image (the frames J > O carry xi = 0: a trail)."""
    c = synth.make_clip("exact_shift", 48, 20, 9, seed=2)
    delta = np.linspace(-0.2, 0.3, c.F).astype(np.float32)
    rgb = c.rgb + delta[:, None, None, None]
    v = oracle.ClipView(rgb, c.depth, c.K, c.w2c)
    O, T = 4, 4
    xi = np.array([0.5 ** (T - j) if j <= T else 0.0 for j in range(2 * T + 1)])
    p = oracle.default_params(c.depth, mode=oracle.MODE_SHUTTER, k=5, T=T, slot_w=xi)
    r = oracle.gather_filter(v, p, O)
    uu = np.arange(c.W)[None, :].repeat(c.H, 0)
    num = np.zeros((c.H, c.W))
    den = np.zeros((c.H, c.W))
    for j in range(2 * T + 1):
        J = O - T + j
        inside = (uu - (J - O) >= 0) & (uu - (J - O) < c.W)
        num += inside * xi[j] * delta[J]
        den += inside * xi[j]
    want = c.rgb[O].astype(np.float64) + (num / den)[..., None]
    np.testing.assert_allclose(r.rgb, want, atol=1e-6, rtol=0)  # float32 offsets
