"""GPU parity of the staged window gather (SSVP_GATHER_WINDOW_TMA): the candidate depths of each
warp's radius tests come from shared-memory boxes filled by TMA tensor copies.  It must gather the
same samples as the window gather that reads the global planes, so it is compared with the FP64
oracle (membership except the radius and tie bands, colour within 1e-3) and, bit for bit, with
SSVP_GATHER_WINDOW on the same inputs, including the 1080p +-30 launch of the benchmark."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import COLOUR_TOL, Session, compare, oracle_params

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


def _staged_and_plain(sess, cid, O, crop=None, membership=True, **kw):
    ss = sess.ss
    a = sess.run(cid, O, crop=crop, membership=membership, gather=ss.SSVP_GATHER_WINDOW_TMA, **kw)
    b = sess.run(cid, O, crop=crop, membership=membership, gather=ss.SSVP_GATHER_WINDOW, **kw)
    np.testing.assert_array_equal(a.rgb, b.rgb)
    if membership:
        np.testing.assert_array_equal(a.status, b.status)
        np.testing.assert_array_equal(a.centre, b.centre)
        np.testing.assert_array_equal(a.bits, b.bits)
        np.testing.assert_array_equal(a.nacc, b.nacc)
        np.testing.assert_array_equal(a.nexam, b.nexam)
        np.testing.assert_array_equal(a.sumw, b.sumw)
    return a


def _box_fit(g, k):
    """Fraction of gathered (pixel, frame) windows that lie inside a 48 x 12 box placed, as the
    kernel places it, around the window of the first gathering lane of their warp (from the
    window centres the GPU records; the kernel's own anchor may differ from them by a pixel)."""
    h = (k - 1) // 2
    ch, cw, ns = g.status.shape
    fit = tot = 0
    for y in range(ch):
        for x0 in range(0, cw, 32):
            st = g.status[y, x0:x0 + 32]
            cen = g.centre[y, x0:x0 + 32]
            for j in range(ns):
                on = np.flatnonzero(st[:, j] == 1)
                if on.size == 0:
                    continue
                lead = on[0]
                ax, ay = cen[lead, j]
                bx = (ax - lead - h + 32 - (48 - 34 - k) // 2) & ~3
                by = ay - h + 32 - (12 - k) // 2
                ox = cen[on, j, 0] - h + 32 - bx
                oy = cen[on, j, 1] - h + 32 - by
                fit += int(((ox >= 0) & (ox <= 48 - k) & (oy >= 0) & (oy <= 12 - k)).sum())
                tot += on.size
    return fit / max(tot, 1)


@pytest.mark.parametrize("O", [0, 7, 15])
def test_staged_tiny_full_frame(sess, O):
    clip = synth.make_clip("planes3", 160, 90, 16, seed=0)
    sess.load(0, clip)
    g = _staged_and_plain(sess, 0, O, k=5, half_window=15)
    med = oracle.median_depth(clip.depth)
    o = oracle.gather_filter(oracle.ClipView.of(clip), oracle_params(med, 5, 15), O, membership=True)
    s = compare(g, o, 5)
    assert s["members"] > 5 * s["pixels"]


def test_staged_hd_crop_and_box_fit(sess):
    clip = synth.make_clip("room", 1280, 720, 60, seed=0)
    sess.load(1, clip)
    crop = (608, 328, 64, 64)
    g = _staged_and_plain(sess, 1, 30, crop=crop, k=7, half_window=15)
    med = oracle.median_depth(clip.depth)
    o = oracle.gather_filter(oracle.ClipView.of(clip), oracle_params(med, 7, 15), 30, crop=crop, membership=True)
    compare(g, o, 7)
    frac = _box_fit(g, 7)
    print(f"windows inside their warp's staged box: {frac:.3f}")
    assert frac > 0.5


@pytest.mark.parametrize("k,T", [(1, 0), (3, 2), (5, 10), (7, 3)])
def test_staged_ragged_sizes(sess, k, T):
    clip = synth.make_clip("planes3", 77, 45, 6, seed=5)
    sess.load(2, clip)
    med = oracle.median_depth(clip.depth)
    for O in (0, 3, 5):
        crop = (3, 5, 41, 29)
        g = _staged_and_plain(sess, 2, O, crop=crop, k=k, half_window=T)
        o = oracle.gather_filter(oracle.ClipView.of(clip), oracle_params(med, k, T), O, crop=crop, membership=True)
        compare(g, o, k)


def test_staged_invalid_depths_and_edges(sess):
    """Invalid reference and candidate depths (NaN, 0, negative, inf): lanes without a valid depth
    take no part in their warp's staging; the one-pixel clip has every window on the border."""
    clip = synth.make_clip("planes3", 64, 40, 5, seed=2)
    depth = clip.depth.copy()
    rng = np.random.default_rng(1)
    bad = rng.random(depth.shape) < 0.15
    depth[bad] = np.array([np.nan, 0.0, -2.0, np.inf], np.float32)[rng.integers(0, 4, bad.sum())]
    c = synth.Clip(clip.W, clip.H, clip.F, clip.K, clip.w2c, clip.w2c_true, clip.rgb, depth, clip.clean,
                   clip.depth_true)
    sess.load(3, c)
    g = _staged_and_plain(sess, 3, 2, k=5, half_window=2)
    o = oracle.gather_filter(oracle.ClipView.of(c), oracle_params(oracle.median_depth(depth), 5, 2), 2,
                             membership=True)
    compare(g, o, 5)
    one = synth.make_clip("planes3", 1, 1, 4, seed=3)
    sess.load(4, one)
    for O in range(one.F):
        g1 = _staged_and_plain(sess, 4, O, k=3, half_window=2)
        np.testing.assert_array_equal(g1.rgb, one.rgb[O])


def test_staged_fp16_colour_and_modes(sess):
    clip = synth.make_clip("planes3", 160, 90, 16, seed=0)
    sess.load(5, clip, colour_fmt=1)
    _staged_and_plain(sess, 5, 8, k=5, half_window=15)
    sess.load(6, clip)
    _staged_and_plain(sess, 6, 8, k=5, half_window=4, mode=sess.ss.SSVP_MODE_MEAN)
    _staged_and_plain(sess, 6, 8, k=7, half_window=127)  # slots outside the clip: no copies


def test_staged_full_size_benchmark_launch(sess):
    """The 1080p +-30, k = 7 launch of the benchmark: the whole output frame equal to the window
    gather's, sampled crops against the oracle."""
    clip = synth.make_clip("room", 1920, 1080, 61, seed=0)
    sess.load(7, clip)
    O = 30
    g = _staged_and_plain(sess, 7, O, membership=False, k=7, half_window=30)
    med = oracle.median_depth(clip.depth)
    v = oracle.ClipView.of(clip)
    for crop in [(0, 0, 24, 24), (960, 540, 24, 24), (1896, 1056, 24, 24)]:
        x0, y0, cw, ch = crop
        o = oracle.gather_filter(v, oracle_params(med, 7, 30), O, crop=crop, membership=True)
        band = ((o.codes & oracle.CODE_BAND) != 0).any(axis=(-1, -2, -3)) | ((o.amb == 1) & (o.status == 1)).any(-1)
        err = np.abs(g.rgb[y0:y0 + ch, x0:x0 + cw] - o.rgb).max(-1)
        assert err[~band].max() <= COLOUR_TOL


def test_staged_argument_errors(sess):
    ss = sess.ss
    clip = synth.make_clip("planes3", 64, 40, 5, seed=2)
    sess.load(8, clip)
    for kw in (dict(k=9), dict(mode=ss.SSVP_MODE_APERTURE), dict(mode=ss.SSVP_MODE_LEARNED)):
        with pytest.raises(ss.SsvpError) as e:
            sess.run(8, 2, gather=ss.SSVP_GATHER_WINDOW_TMA, **kw)
        assert e.value.code == ss.SSVP_EINVAL
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_plan_create(sess.ctx, sess.params(gather=ss.SSVP_GATHER_WINDOW_TMA, frame_begin=1, frame_end=2), [8])
    assert e.value.code == ss.SSVP_EINVAL


def test_staged_copy_wait_time_out(sess):
    """test_skip_mma = 1: the staged gather issues no copies, so every warp's first wait runs out
    (bounded, about 1 s, then 2 s more for copies that might be in flight); ssvp_sync reports
    SSVP_ETIMEOUT, the warps fell back to the global planes (the output equals the window gather's),
    and the next call on the same context runs normally."""
    ss = sess.ss
    clip = synth.make_clip("planes3", 160, 90, 16, seed=0)
    sess.load(9, clip)
    crop = (16, 8, 64, 16)
    want = sess.run(9, 8, crop=crop, k=5, half_window=3).rgb
    t = sess.torch
    p = sess.params(frame_begin=8, frame_end=9, crop_x=crop[0], crop_y=crop[1], crop_w=crop[2], crop_h=crop[3], k=5,
                    half_window=3, gather=ss.SSVP_GATHER_WINDOW_TMA, test_skip_mma=1)
    ss.ssvp_gather_filter(sess.ctx, p, [9])
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_sync(sess.ctx)
    assert e.value.code == ss.SSVP_ETIMEOUT and "tensor-copy" in str(e.value)
    out = t.empty((1, clip.H, clip.W, 3), dtype=t.float32, device=sess.dev)
    ss.ssvp_read_output(sess.ctx, 9, 8, 9, out)
    ss.ssvp_sync(sess.ctx)
    x0, y0, cw, ch = crop
    np.testing.assert_array_equal(out[0, y0:y0 + ch, x0:x0 + cw].cpu().numpy(), want)
    g = _staged_and_plain(sess, 9, 8, crop=crop, k=5, half_window=3)
    np.testing.assert_array_equal(g.rgb, want)


def test_staged_frame_weight_modes(sess):
    """Deblurring (Eq. 5) and the shutter (Eq. 10) through the staged gather: identical to the
    window gather, and the deblurred frame against the oracle."""
    ss = sess.ss
    room = synth.make_clip("room", 96, 54, 9, seed=7)
    sess.load(10, room)
    g = _staged_and_plain(sess, 10, 4, k=5, half_window=4, mode=ss.SSVP_MODE_DEBLUR, radius=-0.03)
    g_w = oracle.frame_sharpness(oracle.ClipView.of(room))
    o = oracle.gather_filter(oracle.ClipView.of(room),
                             oracle_params(oracle.median_depth(room.depth), 5, 4, mode=oracle.MODE_DEBLUR,
                                           radius_rel=0.03, frame_w=g_w / g_w.max()), 4, membership=True)
    compare(g, o, 5)
    xi = np.array([0.5 ** abs(4 - j) for j in range(9)], np.float32)
    ss.ssvp_set_shutter(sess.ctx, xi, 4)
    _staged_and_plain(sess, 10, 4, k=7, half_window=4, mode=ss.SSVP_MODE_SHUTTER)


def test_staged_gather_after_streaming_appends(sess):
    """After ssvp_append_frames the clip's planes live in its second window: the staged gather
    copies from the planes of the current window (its tensor map is made per launch)."""
    ss, t = sess.ss, sess.torch
    W, H, F, N = 96, 54, 9, 3
    video = synth.make_clip("room", W, H, F + 2 * N, seed=6)
    sl = slice(0, F)
    sess.load(11, synth.Clip(W, H, F, video.K[sl], video.w2c[sl], video.w2c_true[sl], video.rgb[sl],
                             video.depth[sl], video.clean[sl], video.depth_true[sl]))
    for i in range(2):
        new = slice(F + i * N, F + (i + 1) * N)
        ss.ssvp_append_frames(sess.ctx, 11, N, np.ascontiguousarray(video.rgb[new]),
                              np.ascontiguousarray(video.depth[new]), video.K[new], 1, video.w2c[new])
        for O in (2, F - 1):
            _staged_and_plain(sess, 11, O, membership=False, k=7, half_window=4)
