"""GPU parity of the frustum gather (Sec. "Sample Gathering", Eq. 1-2) through the C ABI.

Per (pixel, window frame) the sample count and an order-free checksum of the sampled pixels
must equal the FP64 oracle's, except where the oracle saw a candidate within 1e-3 px of Eq. 2's
L1 bound (or within 1e-5 relative of near / far); colour within 1e-3 max abs at every pixel
where no such difference occurred.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import COLOUR_TOL, Session, compare_frustum, run_frustum

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


def _oprm(clip, T, mode, l=3.0, sigma_rel=0.03, **kw):
    med = oracle.median_depth(clip.depth)
    p = oracle.Params(mode=mode, k=1, T=T, radius=0.005 * med, sigma_xyz=sigma_rel * med, gather=oracle.GATHER_FRUSTUM,
                      frustum_l=l, **kw)
    return p, med


def _both(sess, clip, cid, O, T, mode=0, l=3.0, crop=None, near=0.01, far=1000.0):
    p, med = _oprm(clip, T, mode, l, near_plane=near, far_plane=far)
    g = run_frustum(sess, cid, O, crop=crop, membership=True, half_window=T, mode=mode, frustum_l=l,
                    sigma_xyz=p.sigma_xyz, near_plane=near, far_plane=far)
    o = oracle.frustum_filter(oracle.ClipView.of(clip), p, O, crop=crop, membership=True)
    x0, y0, cw, ch = crop if crop is not None else (0, 0, clip.W, clip.H)
    d = clip.depth[O, y0:y0 + ch, x0:x0 + cw]
    return g, o, np.isfinite(d) & (d > 0)


@pytest.mark.parametrize("l", [1.0, 3.0, 5.0])
def test_exact_shift_sets(sess, l):
    c = synth.make_clip("exact_shift", 40, 24, 7, seed=1)
    sess.load(0, c)
    g, o, valid = _both(sess, c, 0, 3, 3, mode=3, l=l)
    s = compare_frustum(g, o, valid)
    assert s["excluded"] == 0 and s["band_slots"] == 0
    # every window frame lies in the clip; frames with samples were scanned (status 1), the rest
    # saw the frustum miss the image (status 0)
    assert np.isin(g.status, (0, 1)).all()
    assert (g.status[g.count > 0] == 1).all()


def test_room_denoise_with_invalid_depths(sess):
    c = synth.make_clip("room", 96, 54, 9, seed=2)
    c.depth[4, 10:14, 20:30] = np.nan   # reference frame holes: c_ref, no samples
    c.depth[2, 30:40, 50:70] = -1.0     # sample-frame holes: never gathered
    c.depth[6, :, :8] = np.inf
    sess.load(1, c)
    g, o, valid = _both(sess, c, 1, 4, 4, mode=0)
    s = compare_frustum(g, o, valid)
    print("room 96x54 frustum:", s)
    assert s["excluded"] <= 0.01 * s["pixels"] + 2
    assert s["members"] > 10 * s["pixels"]


def test_fp16_colour(sess):
    c = synth.make_clip("room", 96, 54, 9, seed=3)
    sess.load(2, c, colour_fmt=1)
    c16 = synth.Clip(c.W, c.H, c.F, c.K, c.w2c, c.w2c_true, c.rgb.astype(np.float16).astype(np.float32), c.depth,
                     c.clean, c.depth_true)
    g, o, valid = _both(sess, c16, 2, 4, 4, mode=0)
    compare_frustum(g, o, valid)


def test_ragged_crop_near_far_and_window_past_the_clip(sess):
    c = synth.make_clip("room", 200, 120, 11, seed=4)
    sess.load(3, c)
    med = oracle.median_depth(c.depth)
    # near and far planes that cut the scene; T reaches past both ends of the clip
    g, o, valid = _both(sess, c, 3, 2, 6, mode=0, crop=(37, 21, 70, 19), near=0.8 * med, far=1.3 * med)
    s = compare_frustum(g, o, valid)
    assert s["excluded"] <= 0.01 * s["pixels"] + 2
    ns = 13
    outside = np.array([not (0 <= 2 - 6 + j < c.F) for j in range(ns)])
    assert (g.status[valid][:, outside] == -1).all()
    assert (g.count[:, :, outside] == 0).all()


def test_hd_full_frame_sampled_against_oracle(sess):
    """1280x720, +-15 frames, the benchmark's launch (whole output frame, no debug outputs);
    sampled crops compared with the oracle, membership through a debug launch of each crop."""
    c = synth.make_clip("room", 1280, 720, 31, seed=0)
    sess.load(4, c)
    O, T = 15, 15
    p, med = _oprm(c, T, 0)
    g = run_frustum(sess, 4, O, half_window=T, mode=0, sigma_xyz=p.sigma_xyz)
    v = oracle.ClipView.of(c)
    for crop in [(0, 0, 4, 4), (640, 360, 4, 4), (1276, 716, 4, 4)]:
        x0, y0, cw, ch = crop
        o = oracle.frustum_filter(v, p, O, crop=crop, membership=True)
        gc = run_frustum(sess, 4, O, crop=crop, membership=True, half_window=T, mode=0, sigma_xyz=p.sigma_xyz)
        d = c.depth[O, y0:y0 + ch, x0:x0 + cw]
        compare_frustum(gc, o, np.isfinite(d) & (d > 0))
        band = o.band.any(-1)
        err = np.abs(g.rgb[y0:y0 + ch, x0:x0 + cw] - o.rgb).max(-1)
        assert err[~band].max(initial=0.0) <= COLOUR_TOL
        np.testing.assert_allclose(g.rgb[y0:y0 + ch, x0:x0 + cw], gc.rgb, atol=1e-6, rtol=0)  # same arithmetic


def test_argument_errors(sess):
    c = synth.make_clip("planes3", 32, 18, 3, seed=0)
    sess.load(5, c)
    ss = sess.ss
    for kw in [dict(frustum_l=0.0), dict(frustum_l=65.0), dict(near_plane=0.0), dict(near_plane=2.0, far_plane=1.0),
               dict(mode=ss.SSVP_MODE_APERTURE), dict(gather=7)]:
        p = sess.params(**{"gather": ss.SSVP_GATHER_FRUSTUM, **kw})
        with pytest.raises(ss.SsvpError) as e:
            ss.ssvp_gather_filter(sess.ctx, p, [5])
        assert e.value.code == ss.SSVP_EINVAL
