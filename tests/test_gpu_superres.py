"""GPU parity of super-resolution (Sec. "Super resolution", Eq. 6-7) through the C ABI against
the FP64 oracle: per (output-grid pixel, window frame) sample counts and membership checksums
exact except within 1e-3 px of Eq. 2's bound, colour within 1e-3 elsewhere."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import COLOUR_TOL, Session, compare_frustum, run_superres
from _gpu import superres_ref_valid as _ref_valid

pytestmark = pytest.mark.gpu


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


def _oprm(c, T, mode=0, l=3.0):
    med = oracle.median_depth(c.depth)
    return oracle.Params(mode=mode, k=1, T=T, radius=0.005 * med, sigma_rgb=50.0 / 255.0, sigma_xyz=0.03 * med,
                         gather=oracle.GATHER_FRUSTUM, frustum_l=l)


def _both(sess, c, cid, O, T, scale, mode=0, l=3.0, crop=None):
    p = _oprm(c, T, mode, l)
    g = run_superres(sess, cid, O, scale, crop=crop, membership=True, half_window=T, mode=mode, frustum_l=l,
                     sigma_rgb=p.sigma_rgb, sigma_xyz=p.sigma_xyz)
    o = oracle.superres_filter(oracle.ClipView.of(c), p, O, scale, crop=crop, membership=True)
    return g, o


@pytest.mark.parametrize("scale", [2, 3])
def test_single_frame_is_bilinear(sess, scale):
    c = synth.make_clip("room", 36, 20, 3, seed=2)
    sess.load(0, c)
    g, o = _both(sess, c, 0, 1, 0, scale, mode=3, l=1.0)
    np.testing.assert_allclose(g.rgb, o.rgb, atol=1e-5, rtol=0)
    np.testing.assert_array_equal(g.nacc, o.nacc)


@pytest.mark.parametrize("scale,cfmt", [(2, 0), (3, 0), (3, 1)])
def test_room_parity(sess, scale, cfmt):
    c = synth.make_clip("room", 48, 27, 7, seed=5)
    c.depth[3, 5:8, 10:16] = np.nan  # holes in the reference frame invalidate nearby references
    if cfmt == 1:
        c = synth.Clip(c.W, c.H, c.F, c.K, c.w2c, c.w2c_true, c.rgb.astype(np.float16).astype(np.float32), c.depth,
                       c.clean, c.depth_true)
    sess.load(1, c, colour_fmt=cfmt)
    g, o = _both(sess, c, 1, 3, 3, scale)
    s = compare_frustum(g, o, _ref_valid(c, 3, scale, None))
    assert s["excluded"] <= 0.01 * s["pixels"] + 2
    assert s["members"] > 2 * s["pixels"]


def test_exact_shift(sess):
    c = synth.make_clip("exact_shift", 24, 12, 7, seed=3)
    sess.load(2, c)
    g, o = _both(sess, c, 2, 3, 3, 3, mode=3)
    s = compare_frustum(g, o, _ref_valid(c, 3, 3, None))
    assert s["excluded"] == 0


def test_ragged_crop(sess):
    c = synth.make_clip("room", 100, 60, 5, seed=6)
    sess.load(3, c)
    crop = (37, 21, 70, 19)
    g, o = _both(sess, c, 3, 2, 2, 2, crop=crop)
    s = compare_frustum(g, o, _ref_valid(c, 2, 2, crop))
    assert s["excluded"] <= 0.01 * s["pixels"] + 2


def test_640x360_to_1080p_sampled(sess):
    """The benchmark's launch (whole 1920x1080 output grid, no debug outputs) from 640x360 input,
    +-15 frames; sampled crops against the oracle and a debug launch of each crop."""
    c = synth.make_clip("room", 640, 360, 31, seed=0)
    sess.load(4, c)
    O, T, s = 15, 15, 3
    p = _oprm(c, T)
    g = run_superres(sess, 4, O, s, half_window=T, sigma_rgb=p.sigma_rgb, sigma_xyz=p.sigma_xyz)
    v = oracle.ClipView.of(c)
    for crop in [(0, 0, 4, 4), (960, 540, 4, 4), (1916, 1076, 4, 4)]:
        x0, y0, cw, ch = crop
        o = oracle.superres_filter(v, p, O, s, crop=crop, membership=True)
        gc = run_superres(sess, 4, O, s, crop=crop, membership=True, half_window=T, sigma_rgb=p.sigma_rgb,
                          sigma_xyz=p.sigma_xyz)
        compare_frustum(gc, o, _ref_valid(c, O, s, crop))
        band = o.band.any(-1)
        err = np.abs(g.rgb[y0:y0 + ch, x0:x0 + cw] - o.rgb).max(-1)
        assert err[~band].max(initial=0.0) <= COLOUR_TOL
        np.testing.assert_allclose(g.rgb[y0:y0 + ch, x0:x0 + cw], gc.rgb, atol=1e-6, rtol=0)


def test_argument_errors(sess):
    c = synth.make_clip("planes3", 32, 18, 3, seed=0)
    sess.load(5, c)
    ss, t = sess.ss, sess.torch
    out = t.zeros((1, 18 * 9, 32 * 9, 3), dtype=t.float32, device=sess.dev)
    for scale, kw in [(0, {}), (9, {}), (2, dict(mode=ss.SSVP_MODE_APERTURE)), (2, dict(frustum_l=0.0)),
                      (2, dict(crop_x=60, crop_y=0, crop_w=10, crop_h=4))]:
        p = sess.params(frame_begin=1, frame_end=2, **kw)
        with pytest.raises(ss.SsvpError) as e:
            ss.ssvp_superres(sess.ctx, p, 5, scale, out)
        assert e.value.code == ss.SSVP_EINVAL
