"""GPU parity of the per-frame weights through the C ABI: deblurring (Sec. "Deblurring", Eq. 5)
and the computational shutter (Sec. "Computational scene-space shutters", Eq. 10), with the
window gather and with the frustum gather, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import COLOUR_TOL, Session, compare, compare_frustum, oracle_params, run_frustum

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


@pytest.fixture(scope="module")
def room():
    c = synth.make_clip("room", 96, 54, 9, seed=7)
    c.rgb[6] = 0.45  # a frame without any gradient: Eq. 5 gives its samples weight 0
    return c


def test_blurriness_sums_match_the_oracle(sess, room):
    sess.load(0, room)
    got = sess.ss.ssvp_frame_sharpness(sess.ctx, 0, room.F)
    want = oracle.frame_sharpness(oracle.ClipView.of(room))
    assert got[6] == 0.0 and want[6] == 0.0
    np.testing.assert_allclose(got, want, rtol=1e-5)
    sess.load(1, room, colour_fmt=1)
    got16 = sess.ss.ssvp_frame_sharpness(sess.ctx, 1, room.F)
    want16 = oracle.frame_sharpness(oracle.ClipView(room.rgb.astype(np.float16).astype(np.float32), room.depth,
                                                    room.K, room.w2c))
    np.testing.assert_allclose(got16, want16, rtol=1e-5)


def test_deblur_window_gather(sess, room):
    sess.load(0, room)
    med = oracle.median_depth(room.depth)
    # the library scales Eq. 5's factor by 1 / max over frames (it cancels in Eq. 3); the oracle
    # gets the same scale so that the sums of weights compare too
    g_w = oracle.frame_sharpness(oracle.ClipView.of(room))
    g_w = g_w / g_w.max()
    for O in (4, 1):
        g = sess.run(0, O, membership=True, k=5, half_window=4, mode=sess.ss.SSVP_MODE_DEBLUR, radius=-0.03)
        o = oracle.gather_filter(oracle.ClipView.of(room), oracle_params(med, 5, 4, mode=oracle.MODE_DEBLUR,
                                                                         radius_rel=0.03, frame_w=g_w), O,
                                 membership=True)
        s = compare(g, o, 5)
        assert s["members"] > 3 * s["pixels"]


def test_shutter_window_gather_closed_form_and_box(sess):
    c = synth.make_clip("exact_shift", 48, 20, 9, seed=2)
    delta = np.linspace(-0.2, 0.3, c.F).astype(np.float32)
    rgb = c.rgb + delta[:, None, None, None]
    sess.load(2, c, rgb=rgb)
    O, T = 4, 4
    xi = np.array([0.5 ** (T - j) if j <= T else 0.0 for j in range(2 * T + 1)], np.float32)
    sess.ss.ssvp_set_shutter(sess.ctx, xi, T)
    g = sess.run(2, O, membership=True, k=5, half_window=T, mode=sess.ss.SSVP_MODE_SHUTTER)
    v = oracle.ClipView(rgb, c.depth, c.K, c.w2c)
    o = oracle.gather_filter(v, oracle_params(oracle.median_depth(c.depth), 5, T, mode=oracle.MODE_SHUTTER,
                                              slot_w=xi.astype(np.float64)), O, membership=True)
    compare(g, o, 5)
    uu = np.arange(c.W)[None, :].repeat(c.H, 0)
    num = sum(((uu - (J - O) >= 0) & (uu - (J - O) < c.W)) * xi[J - O + T] * delta[J] for J in range(O - T, O + T + 1))
    den = sum(((uu - (J - O) >= 0) & (uu - (J - O) < c.W)) * xi[J - O + T] for J in range(O - T, O + T + 1))
    np.testing.assert_allclose(g.rgb, c.rgb[O] + (num / den)[..., None], atol=COLOUR_TOL, rtol=0)
    # a box shutter is the plain average, bit for bit (w = 2^-0 = 1 for every sample)
    sess.ss.ssvp_set_shutter(sess.ctx, np.ones(2 * T + 1, np.float32), T)
    box = sess.run(2, O, k=5, half_window=T, mode=sess.ss.SSVP_MODE_SHUTTER)
    mean = sess.run(2, O, k=5, half_window=T, mode=sess.ss.SSVP_MODE_MEAN)
    np.testing.assert_array_equal(box.rgb, mean.rgb)


@pytest.mark.parametrize("mode", ["deblur", "shutter"])
def test_frustum_gather_with_frame_weights(sess, room, mode):
    sess.load(3, room)
    med = oracle.median_depth(room.depth)
    T, O = 4, 4
    kw = dict(half_window=T, sigma_xyz=0.03 * med)
    p = oracle.Params(k=1, T=T, radius=0.005 * med, sigma_xyz=0.03 * med, gather=oracle.GATHER_FRUSTUM)
    if mode == "deblur":
        kw["mode"] = sess.ss.SSVP_MODE_DEBLUR
        g_w = oracle.frame_sharpness(oracle.ClipView.of(room))
        p.mode, p.frame_w = oracle.MODE_DEBLUR, g_w / g_w.max()  # the library's scale (cancels in Eq. 3)
    else:
        xi = np.array([0.0, 0.25, 0.5, 1.0, 1.0, 1.0, 0.5, 0.25, 0.0], np.float32)
        sess.ss.ssvp_set_shutter(sess.ctx, xi, T)
        kw["mode"] = sess.ss.SSVP_MODE_SHUTTER
        p.mode, p.slot_w = oracle.MODE_SHUTTER, xi.astype(np.float64)
    g = run_frustum(sess, 3, O, membership=True, **kw)
    o = oracle.frustum_filter(oracle.ClipView.of(room), p, O, membership=True)
    d = room.depth[O]
    s = compare_frustum(g, o, np.isfinite(d) & (d > 0))
    assert s["excluded"] <= 0.01 * s["pixels"] + 2


def test_shutter_argument_errors(sess, room):
    sess.load(4, room)
    ss = sess.ss
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_set_shutter(sess.ctx, np.array([1.0, -1.0, 1.0], np.float32), 1)
    assert e.value.code == ss.SSVP_EINVAL
    with pytest.raises(ss.SsvpError):
        ss.ssvp_set_shutter(sess.ctx, np.array([1.0, np.nan, 1.0], np.float32), 1)
    ss.ssvp_set_shutter(sess.ctx, np.ones(3, np.float32), 1)
    with pytest.raises(ss.SsvpError) as e:  # the table covers T = 1, the call asks for T = 2
        ss.ssvp_gather_filter(sess.ctx, sess.params(mode=ss.SSVP_MODE_SHUTTER, half_window=2), [4])
    assert e.value.code == ss.SSVP_EINVAL and "shutter" in str(e.value)
    with pytest.raises(ss.SsvpError) as e:  # batched plans keep to the denoise and mean modes
        ss.ssvp_plan_create(sess.ctx, sess.params(mode=ss.SSVP_MODE_DEBLUR), [4])
    assert e.value.code == ss.SSVP_EINVAL
