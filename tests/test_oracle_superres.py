"""Pins of the oracle's super-resolution (Sec. "Super resolution", Eq. 6-7).

Closed forms used here:
  * at scale 1 with a flat area term the output is the frustum filter's (Eq. 1-4);
  * with T = 0 and l = 1 output pixel, only output pixels whose centre coincides with an input
    pixel centre gather a sample (that pixel itself), so the whole output is the bilinear
    interpolation of the input frame (s_ref) - the reference's definition, pinned against an
    independent numpy bilinear resampler;
  * on the one-pixel-per-frame translation scene, input pixel q of J lands on output
    coordinate scale (q_x + J - O) + (scale - 1) / 2, so the sets are L1 balls in closed form;
  * the area term is a Gaussian in the sample's pixel edge length d / fx (scipy's normal pdf);
  * a rigid motion of the world and all cameras changes nothing.
"""
import numpy as np
import pytest

import oracle
import synth


def _prm(c, T, l=3.0, mode=oracle.MODE_DENOISE, **kw):
    med = oracle.median_depth(c.depth)
    return oracle.Params(mode=mode, k=1, T=T, radius=0.005 * med, sigma_rgb=50.0 / 255.0, sigma_xyz=0.03 * med,
                         gather=oracle.GATHER_FRUSTUM, frustum_l=l, **kw)


def _bilinear_numpy(img, scale):
    """Resample (H, W, C) at u = (U + 0.5) / scale - 0.5 with edge clamping."""
    H, W = img.shape[:2]
    U = (np.arange(W * scale) + 0.5) / scale - 0.5
    V = (np.arange(H * scale) + 0.5) / scale - 0.5
    U, V = np.clip(U, 0, W - 1), np.clip(V, 0, H - 1)
    x0, y0 = np.floor(U).astype(int), np.floor(V).astype(int)
    x1, y1 = np.minimum(x0 + 1, W - 1), np.minimum(y0 + 1, H - 1)
    fx, fy = (U - x0)[None, :, None], (V - y0)[:, None, None]
    im = img.astype(np.float64)
    top = im[y0][:, x0] * (1 - fx) + im[y0][:, x1] * fx
    bot = im[y1][:, x0] * (1 - fx) + im[y1][:, x1] * fx
    return top * (1 - fy) + bot * fy


def test_scale_one_with_flat_area_term_is_the_frustum_filter():
    c = synth.make_clip("room", 40, 24, 7, seed=1)
    v = oracle.ClipView.of(c)
    p = _prm(c, 3)
    a = oracle.superres_filter(v, p, 3, 1, membership=True, sigma_area=1e12)
    b = oracle.frustum_filter(v, p, 3, membership=True)
    ok = ~(a.band.any(-1) | b.band.any(-1))
    assert ok.mean() > 0.9
    np.testing.assert_array_equal(a.count[ok], b.count[ok])
    np.testing.assert_array_equal(a.hash[ok], b.hash[ok])
    np.testing.assert_allclose(a.rgb[ok], b.rgb[ok], atol=1e-12, rtol=0)


@pytest.mark.parametrize("scale", [2, 3])
def test_single_frame_output_is_the_bilinear_reference(scale):
    c = synth.make_clip("room", 36, 20, 3, seed=2)
    v = oracle.ClipView.of(c)
    O = 1
    r = oracle.superres_filter(v, _prm(c, 0, l=1.0, mode=oracle.MODE_MEAN), O, scale, membership=True)
    np.testing.assert_allclose(r.rgb, _bilinear_numpy(c.rgb[O], scale), atol=1e-12, rtol=0)
    # samples only where an output centre coincides with an input centre (odd scale) - one each
    want = np.zeros((c.H * scale, c.W * scale), np.int64)
    if scale % 2 == 1:
        want[scale // 2::scale, scale // 2::scale] = 1
    np.testing.assert_array_equal(r.nacc, want)


def test_exact_shift_sets_on_the_finer_grid():
    c = synth.make_clip("exact_shift", 24, 12, 7, seed=3)
    v = oracle.ClipView.of(c)
    O, T, s, l = 3, 3, 3, 3.0
    r = oracle.superres_filter(v, _prm(c, T, l=l, mode=oracle.MODE_MEAN), O, s, membership=True)
    Hh, Wh = c.H * s, c.W * s
    UU, VV = np.meshgrid(np.arange(Wh), np.arange(Hh))
    qx, qy = np.arange(c.W), np.arange(c.H)
    tot = np.zeros((Hh, Wh))
    n = np.zeros((Hh, Wh), np.int64)
    for j in range(2 * T + 1):
        J = O - T + j
        cx = s * (qx + (J - O)) + (s - 1) / 2  # output-grid coordinate of input pixel q of J
        cy = s * qy + (s - 1) / 2
        d = np.abs(UU[..., None, None] - cx[None, None, None, :]) + np.abs(VV[..., None, None] - cy[None, None, :, None])
        m = d < l / 2  # (Hh, Wh, H, W)
        cnt = m.sum(axis=(-1, -2))
        np.testing.assert_array_equal(r.count[:, :, j], cnt)
        tot += np.einsum("abij,ij->ab", m.astype(np.float64), c.rgb[J][..., 0].astype(np.float64))
        n += cnt
    assert not r.band.any()
    np.testing.assert_array_equal(r.nacc, n)
    has = n > 0
    np.testing.assert_allclose(r.rgb[..., 0][has], (tot / np.maximum(n, 1))[has], atol=1e-12, rtol=0)


def test_area_term_is_a_gaussian_in_the_pixel_edge_length():
    norm = pytest.importorskip("scipy.stats").norm
    s = np.array([0.3, 0.4, 0.5, 1.0, 2.0, 5.0, 3.0])
    sref = s.copy()
    fx, sig = 480.0, 0.01
    for d1, d2 in [(2.0, 4.0), (5.0, 3.0), (7.5, 7.5)]:
        w1 = oracle.weight_superres(s, sref, d1, fx, 0.2, 0.1, 6.0, sig)
        w2 = oracle.weight_superres(s, sref, d2, fx, 0.2, 0.1, 6.0, sig)
        assert w1 / w2 == pytest.approx(norm.pdf(d1 / fx, 0, sig) / norm.pdf(d2 / fx, 0, sig), rel=1e-12)
    # at zero offset to s_ref the Eq. 4 part is 1
    assert oracle.weight_superres(s, sref, 3.0, fx, 0.2, 0.1, 6.0, sig) == pytest.approx(
        norm.pdf(3.0 / fx, 0, sig) / norm.pdf(0, 0, sig), rel=1e-12)


def test_rigid_world_motion_changes_nothing():
    c = synth.make_clip("room", 24, 14, 5, seed=4)
    p = _prm(c, 2)
    a = oracle.superres_filter(oracle.ClipView.of(c), p, 2, 2, membership=True)
    th = 0.4
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    t = np.array([-2.0, 0.5, 1.0])
    w2c = np.empty_like(c.w2c)
    for f in range(c.F):
        w2c[f, :, :3] = c.w2c[f, :, :3] @ R.T
        w2c[f, :, 3] = c.w2c[f, :, 3] - c.w2c[f, :, :3] @ R.T @ t
    b = oracle.superres_filter(oracle.ClipView(c.rgb, c.depth, c.K, w2c), p, 2, 2, membership=True)
    ok = ~(a.band.any(-1) | b.band.any(-1))
    assert ok.mean() > 0.9
    np.testing.assert_array_equal(a.hash[ok], b.hash[ok])
    np.testing.assert_allclose(a.rgb[ok], b.rgb[ok], atol=1e-9, rtol=0)
