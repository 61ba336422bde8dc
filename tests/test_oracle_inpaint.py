"""Pins of the oracle's inpainting (Sec. "Inpainting and semi-transparency", Eq. 8-9).

Closed forms used here, on the exact-geometry scene of constant-albedo planes (the red plane at
depth 3 is the object to remove):
  * the mask of a world box around the red plane is exactly the renderer's own object-id map of
    that plane;
  * where the frustum of a masked pixel sees the background in some frame, the result is the
    background's colour there: the render of the scene without the object (constant planes, so
    every unmasked sample of a uniform neighbourhood has that colour);
  * where it never does, every sample is masked and the result is the mean of S(p) (Eq. 8): the
    object's own colour;
  * an empty mask leaves the frame unchanged.
"""
import numpy as np
import pytest

import oracle
import synth

BOX = (-1.0, -0.7, 2.95, 0.2, 0.3, 3.05)  # world box around the red plane (depth 3) only


@pytest.fixture(scope="module")
def scene():
    c = synth.make_clip("exact_const", 192, 108, 13, seed=0, with_world=True)
    objs = c.meta["objects"]
    bg, _, _, bg_id = synth.render(objs[:2], c.K, c.w2c_true, c.W, c.H, with_world=True)
    return c, bg, bg_id


def _prm(c, T):
    return oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=0.01, sigma_rgb=55.0 / 255.0,
                         gather=oracle.GATHER_FRUSTUM, frustum_l=3.0)


def test_box_mask_is_the_object_id_map(scene):
    c, _, _ = scene
    m = oracle.mask_from_box(oracle.ClipView.of(c), BOX)
    np.testing.assert_array_equal(m.astype(bool), c.objid == 2)
    assert m.sum() > 1000


def test_inpainting_reveals_the_background_or_keeps_the_object(scene):
    c, bg, bg_id = scene
    v = oracle.ClipView.of(c)
    mask = oracle.mask_from_box(v, BOX)
    O, T = 6, 6
    r = oracle.inpaint_filter(v, _prm(c, T), mask, O, membership=True)
    masked = mask[O] == 1
    # unmasked pixels keep their input colour exactly
    np.testing.assert_array_equal(r.rgb[~masked], c.rgb[O][~masked].astype(np.float64))
    # masked pixels whose object-free neighbourhood (9 x 9) is one plane
    pad = np.pad(bg_id[O], 4, mode="edge")
    win = np.lib.stride_tricks.sliding_window_view(pad, (9, 9))
    uniform = (win == bg_id[O][..., None, None]).all(axis=(-1, -2))
    red = c.clean[O][masked][0].astype(np.float64)
    # did an unmasked sample reach the pixel? rebuild from the per-frame counts of an unmasked-only mask
    revealed = np.zeros_like(masked)
    for yy, xx in zip(*np.nonzero(masked & uniform)):
        revealed[yy, xx] = not np.allclose(r.rgb[yy, xx], red, atol=1e-12, rtol=0)
    n_rev, n_hidden = int(revealed.sum()), int((masked & uniform & ~revealed).sum())
    assert n_rev > 50 and n_hidden > 50, (n_rev, n_hidden)
    np.testing.assert_allclose(r.rgb[revealed], bg[O][revealed].astype(np.float64), atol=1e-12, rtol=0)
    np.testing.assert_allclose(r.rgb[masked & uniform & ~revealed], np.broadcast_to(red, (n_hidden, 3)), atol=1e-12,
                               rtol=0)
    # the revealed pixels sit near the object's edge, the hidden ones inside it
    assert r.nacc[masked].min() > 0


def test_empty_mask_changes_nothing(scene):
    c, _, _ = scene
    v = oracle.ClipView.of(c)
    r = oracle.inpaint_filter(v, _prm(c, 3), np.zeros((c.F, c.H, c.W), np.uint8), 6)
    np.testing.assert_array_equal(r.rgb, c.rgb[6].astype(np.float64))
    assert (r.nacc == 0).all()


def test_all_masked_samples_give_the_mean_of_eq8():
    """A pixel whose every sample is masked returns the plain mean of S(p), which on a noisy clip
    is the frustum filter's mean-mode output."""
    c = synth.make_clip("room", 40, 24, 5, seed=3)
    v = oracle.ClipView.of(c)
    p = _prm(c, 2)
    r = oracle.inpaint_filter(v, p, np.ones((c.F, c.H, c.W), np.uint8), 2)
    pm = oracle.Params(**{**p.__dict__, "mode": oracle.MODE_MEAN})
    f = oracle.frustum_filter(v, pm, 2)
    np.testing.assert_allclose(r.rgb, f.rgb, atol=1e-12, rtol=0)
    np.testing.assert_array_equal(r.nacc, f.nacc)
