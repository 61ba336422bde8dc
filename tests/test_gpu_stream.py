"""Streaming video through ssvp_append_frames: after every append the clip must behave exactly
like a fresh load of the same frame window (outputs bit for bit, median, per-frame values), for
host and device inputs, FP32 and FP16 colour, the window and the frustum gathers and the
per-frame (Eq. 5) weights; queued appends must be ordered with the gathers around them."""
import numpy as np
import pytest

import synth
from _gpu import Session

pytestmark = pytest.mark.gpu

W, H, F, N = 96, 54, 9, 3


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
def video():
    return synth.make_clip("room", W, H, F + 7 * N, seed=6)


def _window(v, k0):
    sl = slice(k0, k0 + F)
    return synth.Clip(W, H, F, v.K[sl], v.w2c[sl], v.w2c_true[sl], v.rgb[sl], v.depth[sl], v.clean[sl],
                      v.depth_true[sl])


def _outputs(sess, cid, params):
    t = sess.torch
    res = []
    for kw in params:
        p = sess.params(frame_begin=0, frame_end=F, **kw)
        sess.ss.ssvp_gather_filter(sess.ctx, p, [cid])
        out = t.empty((F, H, W, 3), dtype=t.float32, device=sess.dev)
        sess.ss.ssvp_read_output(sess.ctx, cid, 0, F, out)
        sess.ss.ssvp_sync(sess.ctx)
        res.append(out.cpu().numpy())
    return res


PARAMS = [dict(k=5, half_window=3), dict(k=7, half_window=4, mode=4, sigma_rgb=200 / 255, sigma_f=20.0),
          dict(half_window=2, gather=1, radius=-0.03, sigma_xyz=0.0)]


@pytest.mark.parametrize("cfmt", [0, 1])
def test_appends_equal_fresh_loads_of_the_same_window(sess, video, cfmt):
    t, ss = sess.torch, sess.ss
    sess.load(20, _window(video, 0), colour_fmt=cfmt)
    start = 0  # the clip holds video frames start .. start + F - 1
    for step, n in enumerate((N, N, 2 * N, F)):  # the last one replaces the whole window
        new = slice(start + F, start + F + n)
        rgb, dep = np.ascontiguousarray(video.rgb[new]), np.ascontiguousarray(video.depth[new])
        if step % 2:  # device inputs on every other append
            rgb, dep = t.from_numpy(rgb).to(sess.dev), t.from_numpy(dep).to(sess.dev)
        ss.ssvp_append_frames(sess.ctx, 20, n, rgb, dep, video.K[new], 1, video.w2c[new])
        start += n
        sess.load(21, _window(video, start), colour_fmt=cfmt)
        assert ss.ssvp_clip_median_depth(sess.ctx, 20) == ss.ssvp_clip_median_depth(sess.ctx, 21)
        for a, b in zip(_outputs(sess, 20, PARAMS), _outputs(sess, 21, PARAMS)):
            np.testing.assert_array_equal(a, b)


def test_queued_appends_are_ordered_with_the_gathers(sess, video):
    t, ss = sess.torch, sess.ss
    p = sess.params(k=5, half_window=3, frame_begin=0, frame_end=F)
    want = []
    for k0 in (0, N, 2 * N, 3 * N):
        sess.load(23, _window(video, k0))
        want.append(_outputs(sess, 23, [dict(k=5, half_window=3)])[0])
    sess.load(22, _window(video, 0))
    outs = [t.empty((F, H, W, 3), dtype=t.float32, device=sess.dev) for _ in range(4)]
    ss.ssvp_gather_filter(sess.ctx, p, [22])
    ss.ssvp_read_output(sess.ctx, 22, 0, F, outs[0])
    for i in (1, 2, 3):  # no synchronisation until the end
        new = slice(F + (i - 1) * N, F + i * N)
        ss.ssvp_append_frames(sess.ctx, 22, N, np.ascontiguousarray(video.rgb[new]),
                              np.ascontiguousarray(video.depth[new]), video.K[new], 1, video.w2c[new])
        ss.ssvp_gather_filter(sess.ctx, p, [22])
        ss.ssvp_read_output(sess.ctx, 22, 0, F, outs[i])
    ss.ssvp_sync(sess.ctx)
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)


def test_append_argument_errors(sess, video):
    ss = sess.ss
    sess.load(24, _window(video, 0))
    rgb, dep = np.ascontiguousarray(video.rgb[:2]), np.ascontiguousarray(video.depth[:2])
    for n in (0, F + 1):
        with pytest.raises(ss.SsvpError) as e:
            ss.ssvp_append_frames(sess.ctx, 24, n, rgb, dep, video.K[:2], 1, video.w2c[:2])
        assert e.value.code == ss.SSVP_EINVAL
    bad = video.w2c[:2].copy()
    bad[0, 0, 0] = 2.0  # not a rotation
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_append_frames(sess.ctx, 24, 2, rgb, dep, video.K[:2], 1, bad)
    assert e.value.code == ss.SSVP_EINVAL
    ss.ssvp_mask_from_box(sess.ctx, 24, (-1, -1, 0, 1, 1, 100))
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_append_frames(sess.ctx, 24, 2, rgb, dep, video.K[:2], 1, video.w2c[:2])
    assert e.value.code == ss.SSVP_EINVAL and "mask" in str(e.value)
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_append_frames(sess.ctx, 25, 2, rgb, dep, video.K[:2], 1, video.w2c[:2])
    assert e.value.code == ss.SSVP_ENOCLIP
