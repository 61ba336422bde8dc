"""GPU parity of inpainting (Sec. "Inpainting and semi-transparency", Eq. 8-9) through the C ABI:
the box mask bit for bit, then per (masked pixel, window frame) sample counts and membership
checksums, and colours within 1e-3, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import Session, compare_frustum, run_frustum

pytestmark = pytest.mark.gpu

BOX = (-1.0, -0.7, 2.95, 0.2, 0.3, 3.05)  # around the red plane of the constant-plane scene


@pytest.fixture(scope="module")
def sess():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    s = Session()
    yield s
    s.close()


def _prm(T):
    return oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=0.01, sigma_rgb=55.0 / 255.0,
                         gather=oracle.GATHER_FRUSTUM, frustum_l=3.0)


def _both(sess, c, cid, mask, O, T, crop=None):
    g = run_frustum(sess, cid, O, crop=crop, membership=True, half_window=T, mode=sess.ss.SSVP_MODE_INPAINT,
                    sigma_rgb=55.0 / 255.0)
    o = oracle.inpaint_filter(oracle.ClipView.of(c), _prm(T), mask, O, crop=crop, membership=True)
    x0, y0, cw, ch = crop if crop is not None else (0, 0, c.W, c.H)
    return g, o, mask[O, y0:y0 + ch, x0:x0 + cw] != 0


def test_box_mask_and_inpainting_on_constant_planes(sess):
    c = synth.make_clip("exact_const", 192, 108, 13, seed=0, with_world=True)
    sess.load(0, c)
    sess.ss.ssvp_mask_from_box(sess.ctx, 0, BOX)
    got = sess.ss.ssvp_read_mask(sess.ctx, 0, c.F, c.H, c.W)
    want = oracle.mask_from_box(oracle.ClipView.of(c), BOX)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got.astype(bool), c.objid == 2)
    g, o, masked = _both(sess, c, 0, want, 6, 6)
    s = compare_frustum(g, o, masked)
    assert s["excluded"] == 0
    np.testing.assert_array_equal(g.rgb[~masked], c.rgb[6][~masked])  # untouched outside the mask


def test_room_box_mask(sess):
    c = synth.make_clip("room", 96, 54, 9, seed=0)
    sess.load(1, c)
    box = synth.object_box(c.meta["objects"][9], 0.02, (-2.18, 1.48))
    sess.ss.ssvp_mask_from_box(sess.ctx, 1, box)
    mask = oracle.mask_from_box(oracle.ClipView.of(c), box)
    np.testing.assert_array_equal(sess.ss.ssvp_read_mask(sess.ctx, 1, c.F, c.H, c.W), mask)
    assert mask[4].sum() > 100
    g, o, masked = _both(sess, c, 1, mask, 4, 4)
    s = compare_frustum(g, o, masked)
    assert s["excluded"] <= 0.01 * s["pixels"] + 2


def test_painted_mask_from_the_host_and_a_crop(sess):
    c = synth.make_clip("room", 80, 48, 7, seed=2)
    sess.load(2, c)
    yy, xx = np.mgrid[0:c.H, 0:c.W]
    mask = np.zeros((c.F, c.H, c.W), np.uint8)
    for f in range(c.F):  # a disc drifting across the frames
        mask[f] = ((xx - 30 - 2 * f) ** 2 + (yy - 20) ** 2 < 64).astype(np.uint8)
    sess.ss.ssvp_set_mask(sess.ctx, 2, mask)
    np.testing.assert_array_equal(sess.ss.ssvp_read_mask(sess.ctx, 2, c.F, c.H, c.W), mask)
    g, o, masked = _both(sess, c, 2, mask, 3, 3, crop=(27, 9, 29, 21))
    s = compare_frustum(g, o, masked)
    assert s["excluded"] <= 0.01 * s["pixels"] + 2


def test_argument_errors(sess):
    c = synth.make_clip("planes3", 32, 18, 3, seed=0)
    sess.load(3, c)
    ss = sess.ss
    with pytest.raises(ss.SsvpError) as e:  # no mask yet
        ss.ssvp_gather_filter(sess.ctx, sess.params(mode=ss.SSVP_MODE_INPAINT, gather=ss.SSVP_GATHER_FRUSTUM), [3])
    assert e.value.code == ss.SSVP_EINVAL and "mask" in str(e.value)
    ss.ssvp_mask_from_box(sess.ctx, 3, (-1, -1, 0, 1, 1, 100))
    with pytest.raises(ss.SsvpError) as e:  # inpainting needs the frustum gather
        ss.ssvp_gather_filter(sess.ctx, sess.params(mode=ss.SSVP_MODE_INPAINT), [3])
    assert e.value.code == ss.SSVP_EINVAL
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_mask_from_box(sess.ctx, 3, (0, 0, 0, np.nan, 1, 1))
    assert e.value.code == ss.SSVP_EINVAL


# ---------------------------------------------------------------- semi-transparency (after Eq. 9)
SEMI_SIGMA_RGB = 80.0 / 255.0  # the paper's sigma_rgb = 80 for semi-transparency


def _semi_both(sess, c, cid, mask, O, T, sigma_xyz, crop=None):
    g = run_frustum(sess, cid, O, crop=crop, membership=True, half_window=T, mode=sess.ss.SSVP_MODE_SEMI,
                    sigma_rgb=SEMI_SIGMA_RGB, sigma_xyz=sigma_xyz)
    prm = oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=0.01, sigma_rgb=SEMI_SIGMA_RGB, sigma_xyz=sigma_xyz,
                        gather=oracle.GATHER_FRUSTUM, frustum_l=3.0)
    o = oracle.inpaint_filter(oracle.ClipView.of(c), prm, mask, O, crop=crop, membership=True, semi=True)
    x0, y0, cw, ch = crop if crop is not None else (0, 0, c.W, c.H)
    return g, o, mask[O, y0:y0 + ch, x0:x0 + cw] != 0


def test_semitransparency_on_constant_planes(sess):
    c = synth.make_clip("exact_const", 192, 108, 13, seed=0)
    sess.load(4, c)
    sess.ss.ssvp_mask_from_box(sess.ctx, 4, BOX)
    mask = oracle.mask_from_box(oracle.ClipView.of(c), BOX)
    g, o, masked = _semi_both(sess, c, 4, mask, 6, 6, sigma_xyz=0.05)
    s = compare_frustum(g, o, masked)
    assert s["excluded"] == 0
    np.testing.assert_array_equal(g.rgb[~masked], c.rgb[6][~masked])
    # see-through: revealed pixels differ from both the object's colour and inpainting's result
    gi = run_frustum(sess, 4, 6, half_window=6, mode=sess.ss.SSVP_MODE_INPAINT, sigma_rgb=SEMI_SIGMA_RGB)
    mid = masked & (np.abs(gi.rgb - c.rgb[6]).max(-1) > 0.05)
    assert mid.sum() > 50
    assert (np.abs(g.rgb[mid] - gi.rgb[mid]).max(-1) > 1e-3).all()
    assert (np.abs(g.rgb[mid] - c.rgb[6][mid]).max(-1) > 1e-3).all()


def test_semitransparency_on_the_room_scene_with_invalid_depths(sess):
    c = synth.make_clip("room", 96, 54, 9, seed=0)
    box = synth.object_box(c.meta["objects"][9], 0.02, (-2.18, 1.48))
    mask = oracle.mask_from_box(oracle.ClipView.of(c), box)
    ys, xs = np.nonzero(mask[4])
    depth = c.depth.copy()
    for i in range(0, len(ys), max(1, len(ys) // 5)):  # masked pixels without a valid depth
        depth[4, ys[i], xs[i]] = np.nan
    bad = synth.Clip(c.W, c.H, c.F, c.K, c.w2c, c.w2c_true, c.rgb, depth, c.clean, c.depth_true)
    sess.load(5, bad)
    sess.ss.ssvp_set_mask(sess.ctx, 5, mask)
    med = oracle.median_depth(c.depth)
    g, o, masked = _semi_both(sess, bad, 5, mask, 4, 4, sigma_xyz=0.03 * med)
    s = compare_frustum(g, o, masked)
    assert s["excluded"] <= 0.01 * s["pixels"] + 2


def test_semitransparency_of_a_fully_masked_frame_is_the_eq4_frustum_filter(sess):
    c = synth.make_clip("room", 64, 36, 7, seed=3)
    sess.load(6, c)
    mask = np.ones((c.F, c.H, c.W), np.uint8)
    sess.ss.ssvp_set_mask(sess.ctx, 6, mask)
    sx = 0.02
    g, o, masked = _semi_both(sess, c, 6, mask, 3, 3, sigma_xyz=sx, crop=(5, 3, 41, 29))
    compare_frustum(g, o, masked)
    f = run_frustum(sess, 6, 3, crop=(5, 3, 41, 29), half_window=3, sigma_rgb=SEMI_SIGMA_RGB, sigma_xyz=sx)
    assert np.abs(g.rgb - f.rgb).max() <= 1e-5


def test_reload_keeps_the_mask_and_box_masks_queue_without_waiting(sess):
    """A reload with the same shape keeps the mask (and its memory); masks from two boxes queued
    back to back, each followed by a gather, give each gather its own mask."""
    c = synth.make_clip("exact_const", 96, 54, 9, seed=0)
    sess.load(7, c)
    sess.ss.ssvp_mask_from_box(sess.ctx, 7, BOX)
    want = oracle.mask_from_box(oracle.ClipView.of(c), BOX)
    sess.load(7, c)  # same shape and format: planes and mask kept
    np.testing.assert_array_equal(sess.ss.ssvp_read_mask(sess.ctx, 7, c.F, c.H, c.W), want)
    g1, o1, masked = _both(sess, c, 7, want, 4, 4)
    assert masked.sum() > 20
    s = compare_frustum(g1, o1, masked)
    assert s["excluded"] == 0
    box2 = (-10.0, -10.0, 0.0, 10.0, 10.0, 100.0)  # everything with a valid depth
    want2 = oracle.mask_from_box(oracle.ClipView.of(c), box2)
    assert want2.sum() > want.sum()
    sess.ss.ssvp_mask_from_box(sess.ctx, 7, BOX)
    sess.ss.ssvp_mask_from_box(sess.ctx, 7, box2)
    np.testing.assert_array_equal(sess.ss.ssvp_read_mask(sess.ctx, 7, c.F, c.H, c.W), want2)
