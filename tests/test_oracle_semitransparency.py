"""Pins of the oracle's semi-transparency (Sec. "Inpainting and semi-transparency", the variant
after Eq. 9: the input frame's own sample adds the standard multivariate weighting of Eq. 4).

The reading: inpainting's Eq. 8 mean and first Eq. 9 step, then a second step in which every
sample s of S(p) weighs [M(s) = 0] exp(-|c_ref - c_s|^2 / (2 sigma_rgb^2)) + w_Eq4(s; s_I), with
s_I = (I_O(p), x_ref, O) the pixel's own sample.  Checks against independent results:
  * a frame whose every pixel is masked has no background term: the output is the frustum
    gather's Eq. 4 filter (around the pixel's own sample) exactly;
  * with sigma_xyz -> 0 only the pixel's own sample keeps its Eq. 4 weight (1): the output is
    inpainting's result blended with I(p) by their weights, (W_inp inp + I(p)) / (W_inp + 1),
    from the inpainting oracle's own output and sum of weights;
  * with every sigma -> infinity all weights are 1: (N mean(S) + N_u mean(unmasked)) / (N + N_u),
    from the frustum mean filter (N, mean(S)) and inpainting (N_u = its sum of weights);
  * unmasked pixels, an empty mask and a masked pixel without a valid depth behave as in
    inpainting.
"""
import numpy as np
import pytest

import oracle
import synth

BOX = (-1.0, -0.7, 2.95, 0.2, 0.3, 3.05)  # world box around the red plane (depth 3) of exact_const


@pytest.fixture(scope="module")
def scene():
    c = synth.make_clip("exact_const", 192, 108, 13, seed=0)
    v = oracle.ClipView.of(c)
    return c, v, oracle.mask_from_box(v, BOX)


@pytest.fixture(scope="module")
def room():
    c = synth.make_clip("room", 48, 27, 7, seed=4)
    return c, oracle.ClipView.of(c)


def _prm(T, sigma_rgb=80.0 / 255.0, sigma_xyz=0.05, sigma_f=6.0, mode=oracle.MODE_DENOISE):
    return oracle.Params(mode=mode, k=1, T=T, radius=0.01, sigma_rgb=sigma_rgb, sigma_xyz=sigma_xyz, sigma_f=sigma_f,
                         gather=oracle.GATHER_FRUSTUM, frustum_l=3.0)


def test_all_masked_is_the_frustum_eq4_filter(room):
    c, v = room
    p = _prm(3, sigma_xyz=0.03)
    r = oracle.inpaint_filter(v, p, np.ones((c.F, c.H, c.W), np.uint8), 3, semi=True)
    f = oracle.frustum_filter(v, p, 3)
    np.testing.assert_allclose(r.rgb, f.rgb, atol=1e-12, rtol=0)
    np.testing.assert_array_equal(r.nacc, f.nacc)
    # and it differs from plain inpainting (the Eq. 8 mean): the Eq. 4 term does the work
    i = oracle.inpaint_filter(v, p, np.ones((c.F, c.H, c.W), np.uint8), 3)
    assert np.abs(i.rgb - r.rgb).max() > 1e-3


def test_tiny_sigma_xyz_blends_inpainting_with_the_input_pixel(scene):
    c, v, mask = scene
    O, T = 6, 6
    p = _prm(T, sigma_xyz=1e-9)
    s = oracle.inpaint_filter(v, p, mask, O, semi=True)
    i = oracle.inpaint_filter(v, p, mask, O)
    m = mask[O] == 1
    I = c.rgb[O].astype(np.float64)
    want = (i.sumw[..., None] * i.rgb + I) / (i.sumw[..., None] + 1.0)
    np.testing.assert_allclose(s.rgb[m], want[m], atol=1e-12, rtol=0)
    np.testing.assert_array_equal(s.rgb[~m], I[~m])
    # revealed pixels (some background weight) end between the object and the background
    rev = m & (i.sumw > 0.5)
    assert rev.sum() > 50
    d_obj, d_inp = np.abs(s.rgb[rev] - I[rev]).max(-1), np.abs(s.rgb[rev] - i.rgb[rev]).max(-1)
    assert (d_obj > 0).all() and (d_inp > 0).all()


def test_infinite_sigmas_weigh_every_sample_once_and_unmasked_twice(scene):
    c, v, mask = scene
    O, T = 6, 4
    big = 1e9
    p = _prm(T, sigma_rgb=big, sigma_xyz=big, sigma_f=big)
    s = oracle.inpaint_filter(v, p, mask, O, semi=True)
    i = oracle.inpaint_filter(v, p, mask, O)
    f = oracle.frustum_filter(v, _prm(T, mode=oracle.MODE_MEAN), O)
    m = mask[O] == 1
    N, Nu = f.nacc[..., None].astype(np.float64), i.sumw[..., None]
    want = (N * f.rgb + Nu * i.rgb) / (N + Nu)
    np.testing.assert_allclose(s.rgb[m], want[m], atol=1e-12, rtol=0)
    np.testing.assert_array_equal(s.nacc[m], f.nacc[m])
    assert (Nu[m] > 0).sum() > 50 and (Nu[m] == 0).sum() > 50


def test_empty_mask_unmasked_pixels_and_invalid_depth(scene, room):
    c, v, mask = scene
    p = _prm(3)
    r = oracle.inpaint_filter(v, p, np.zeros((c.F, c.H, c.W), np.uint8), 6, semi=True)
    np.testing.assert_array_equal(r.rgb, c.rgb[6].astype(np.float64))
    # a masked pixel without a valid depth has no own sample: inpainting's result
    c2, _ = room
    d = c2.depth.copy()
    d[3, 10, 20] = np.nan
    d[3, 5, 7] = -1.0
    v2 = oracle.ClipView(c2.rgb, d, c2.K, c2.w2c)
    full = np.ones((c2.F, c2.H, c2.W), np.uint8)
    full[:, :, :3] = 0  # some unmasked samples
    s = oracle.inpaint_filter(v2, _prm(2), full, 3, semi=True)
    i = oracle.inpaint_filter(v2, _prm(2), full, 3)
    for y, x in ((10, 20), (5, 7)):
        np.testing.assert_array_equal(s.rgb[y, x], i.rgb[y, x])
    assert np.abs(s.rgb - i.rgb).max() > 1e-3


def test_semitransparency_needs_finite_positive_sigmas(room):
    c, v = room
    with pytest.raises(ValueError):
        oracle.inpaint_filter(v, _prm(2, sigma_xyz=0.0), np.ones((c.F, c.H, c.W), np.uint8), 3, semi=True)
