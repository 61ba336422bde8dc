"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Membership must match exactly except candidates within 1e-5 relative of the radius and window
centres within 1e-3 px of a rounding tie; colour within 1e-3 max abs at every other pixel.
"""
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


@pytest.fixture(scope="module")
def tiny():
    # the tiny workload: 160x90, 16 frames, 3 textured planes
    return synth.make_clip("planes3", 160, 90, 16, seed=0)


@pytest.fixture(scope="module")
def hd():
    # the HD workload: 1280x720, 60 frames, 6 planes + 4 boxes, hand-held camera
    return synth.make_clip("room", 1280, 720, 60, seed=0)


def _both(sess, clip, cid, O, k, T, crop=None, colour_fmt=0, mode=0, **kw):
    med = oracle.median_depth(clip.depth)
    g = sess.run(cid, O, crop=crop, membership=True, k=k, half_window=T, mode=mode, **kw)
    o = oracle.gather_filter(oracle.ClipView.of(clip), oracle_params(med, k, T, mode=mode), O, crop=crop,
                             membership=True)
    return g, o


@pytest.mark.parametrize("O", [0, 7, 15])
def test_tiny_full_frame(sess, tiny, O):
    sess.load(0, tiny)
    g, o = _both(sess, tiny, 0, O, k=5, T=15)
    s = compare(g, o, 5)
    assert s["members"] > 5 * s["pixels"]
    assert s["excluded"] <= 0.001 * s["pixels"] + 2


def test_hd_crop(sess, hd):
    sess.load(1, hd)
    g, o = _both(sess, hd, 1, 30, k=7, T=15, crop=(608, 328, 64, 64))
    s = compare(g, o, 7)
    assert s["excluded"] <= 0.001 * s["pixels"] + 2


@pytest.mark.parametrize("k,T", [(1, 0), (3, 2), (9, 1), (31, 1), (5, 10)])
def test_ragged_sizes_and_windows(sess, k, T):
    clip = synth.make_clip("planes3", 77, 45, 6, seed=5)
    sess.load(2, clip)
    for O in (0, 3, 5):
        g, o = _both(sess, clip, 2, O, k=k, T=T, crop=(3, 5, 41, 29))
        compare(g, o, k)


def test_self_reprojection_is_bit_exact(sess, tiny):
    sess.load(0, tiny)
    g = sess.run(0, 4, membership=True, k=1, half_window=0)
    np.testing.assert_array_equal(g.rgb, tiny.rgb[4])
    assert (g.nacc == 1).all()


def test_invalid_depths(sess):
    clip = synth.make_clip("planes3", 64, 40, 5, seed=2)
    depth = clip.depth.copy()
    rng = np.random.default_rng(1)
    bad = rng.random(depth.shape) < 0.15
    depth[bad] = np.array([np.nan, 0.0, -2.0, np.inf], np.float32)[rng.integers(0, 4, bad.sum())]
    bad_clip = synth.Clip(clip.W, clip.H, clip.F, clip.K, clip.w2c, clip.w2c_true, clip.rgb, depth, clip.clean,
                          clip.depth_true)
    sess.load(3, bad_clip)
    g, o = _both(sess, bad_clip, 3, 2, k=5, T=2)
    compare(g, o, 5)
    np.testing.assert_array_equal(g.rgb[bad[2]], clip.rgb[2][bad[2]])


def test_mean_mode(sess, tiny):
    sess.load(0, tiny)
    g, o = _both(sess, tiny, 0, 8, k=5, T=4, mode=3)
    compare(g, o, 5)


def test_fp16_colour(sess, tiny):
    """FP16 colour storage: arithmetic parity against the oracle on the FP16-rounded colours, and
    the total error against the FP32-colour oracle reported (bounded by the FP16 rounding)."""
    sess.load(4, tiny, colour_fmt=1)
    rgb16 = tiny.rgb.astype(np.float16).astype(np.float32)
    c16 = synth.Clip(tiny.W, tiny.H, tiny.F, tiny.K, tiny.w2c, tiny.w2c_true, rgb16, tiny.depth, tiny.clean,
                     tiny.depth_true)
    g, o16 = _both(sess, c16, 4, 8, k=5, T=15)
    compare(g, o16, 5)
    med = oracle.median_depth(tiny.depth)
    o32 = oracle.gather_filter(oracle.ClipView.of(tiny), oracle_params(med, 5, 15), 8)
    # total error of FP16 storage: colour rounding (2^-11 relative) plus its effect on the Eq. 4
    # colour weights of outlying samples; stated, and bounded loosely
    total = float(np.abs(g.rgb - o32.rgb).max())
    print(f"FP16 colour: max |GPU - FP32-colour oracle| = {total:.3e}")
    assert total < 1e-2


def test_exact_geometry_reproduces_clean(sess):
    """Exact depth and poses, constant-albedo planes: the output is the clean render to 1e-6."""
    c = synth.make_clip("exact_const", 96, 54, 9, seed=0)
    sess.load(5, c)
    g = sess.run(5, 4, membership=True, k=5, half_window=4)
    assert np.abs(g.rgb - c.clean[4]).max() <= 1e-6
    assert g.nacc.mean() > 0.5 * c.F


def test_exact_shift_membership_closed_form(sess):
    c = synth.make_clip("exact_shift", 64, 36, 7, seed=1)
    sess.load(6, c)
    O, T, h = 3, 3, 2
    g = sess.run(6, O, membership=True, k=5, half_window=T)
    uu = np.arange(c.W)[None, :].repeat(c.H, 0)
    for j in range(2 * T + 1):
        J = O - T + j
        inside = (uu - (J - O) >= 0) & (uu - (J - O) < c.W)
        assert (g.bits[:, :, j, h, h] == inside).all()
        b = g.bits[:, :, j].copy()
        b[:, :, h, h] = False
        assert not b.any()
    assert np.abs(g.rgb - c.clean[O]).max() <= 1e-6


def test_median_depth_is_exact(sess, tiny):
    sess.load(0, tiny)
    assert sess.ss.ssvp_clip_median_depth(sess.ctx, 0) == oracle.median_depth(tiny.depth)
    d = tiny.depth[:3].copy()
    d[0, :10] = np.nan
    d[1, 5:20] = -1.0
    d[2, :, :7] = 0.0
    c = synth.Clip(tiny.W, tiny.H, 3, tiny.K[:3], tiny.w2c[:3], tiny.w2c_true[:3], tiny.rgb[:3], d, tiny.clean[:3],
                   tiny.depth_true[:3])
    sess.load(7, c)
    assert sess.ss.ssvp_clip_median_depth(sess.ctx, 7) == oracle.median_depth(d)


def test_host_upload_matches_device_upload(sess, tiny):
    sess.load(0, tiny)
    a = sess.run(0, 8, k=5, half_window=15).rgb
    sess.load(8, tiny, host=True)
    b = sess.run(8, 8, k=5, half_window=15).rgb
    np.testing.assert_array_equal(a, b)


def test_reload_with_the_same_shape_replaces_the_contents(sess, tiny):
    """A reload of an id with the same shape keeps the device planes: the new frames, depths,
    cameras and median must replace the old ones completely (also through a host upload)."""
    other = synth.make_clip("room", tiny.W, tiny.H, tiny.F, seed=9)
    sess.load(9, other)
    want_other = sess.run(9, 8, k=5, half_window=15).rgb
    sess.load(9, tiny)  # same W, H, F and format: the planes are reused
    assert sess.ss.ssvp_clip_median_depth(sess.ctx, 9) == oracle.median_depth(tiny.depth)
    sess.load(10, tiny)  # a fresh id for the reference
    np.testing.assert_array_equal(sess.run(9, 8, k=5, half_window=15).rgb, sess.run(10, 8, k=5, half_window=15).rgb)
    sess.load(9, other, host=True)
    np.testing.assert_array_equal(sess.run(9, 8, k=5, half_window=15).rgb, want_other)


def test_reload_clears_every_output_frame_written_since_the_load(sess, tiny):
    """Pixels no gather has written since the (re)load read 0: a same-shape reload clears the
    frames written by gathers, batched plans and the caller through the device pointer."""
    ss, t = sess.ss, sess.torch
    sess.load(14, tiny)
    ss.ssvp_gather_filter(sess.ctx, sess.params(k=5, half_window=2, frame_begin=2, frame_end=4), [14])
    plan = ss.ssvp_plan_create(sess.ctx, sess.params(k=5, half_window=2, frame_begin=9, frame_end=11), [14])
    ss.ssvp_plan_launch(plan)
    ss.ssvp_plan_destroy(plan)
    out = t.empty((tiny.F, tiny.H, tiny.W, 3), dtype=t.float32, device=sess.dev)
    ss.ssvp_read_output(sess.ctx, 14, 0, tiny.F, out)
    ss.ssvp_sync(sess.ctx)
    written = [f for f in range(tiny.F) if bool((out[f] != 0).any())]
    assert written == [2, 3, 9, 10]
    sess.load(14, tiny)  # same shape: planes reused, the written frames cleared
    ss.ssvp_read_output(sess.ctx, 14, 0, tiny.F, out)
    ss.ssvp_sync(sess.ctx)
    assert not bool((out != 0).any())
    # the caller writes the last frame through the device pointer (wrapped without a copy)
    ptr = ss.ssvp_output_device_ptr(sess.ctx, 14)

    class _Buf:
        __cuda_array_interface__ = {"shape": (tiny.F, tiny.H, tiny.W, 3), "typestr": "<f4", "data": (ptr, False),
                                    "version": 2}

    buf = t.as_tensor(_Buf(), device=sess.dev)
    sess.stream.synchronize()
    buf[tiny.F - 1].fill_(2.0)
    t.cuda.synchronize()
    ss.ssvp_read_output(sess.ctx, 14, tiny.F - 1, tiny.F, out[:1])
    ss.ssvp_sync(sess.ctx)
    assert bool((out[0] == 2.0).all())
    sess.load(14, tiny)
    ss.ssvp_read_output(sess.ctx, 14, 0, tiny.F, out)
    ss.ssvp_sync(sess.ctx)
    assert not bool((out != 0).any())


def test_allocation_failure_is_a_status_and_the_context_stays_usable(sess, tiny):
    """A clip whose planes exceed the device (16384 x 16384 x 4096: ~4 TB of depth alone) is refused
    with SSVP_ENOMEM by the first allocation, before any input is read; nothing stays allocated,
    the id is not loaded, and the context goes on working."""
    ss = sess.ss
    host = np.zeros(16, np.float32)  # never read: the allocation fails first
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_load_clip(sess.ctx, 15, 16384, 16384, 4096, host, host, ss.SSVP_MEM_HOST)
    assert e.value.code == ss.SSVP_ENOMEM and "cudaMalloc" in str(e.value)
    with pytest.raises(ss.SsvpError) as e2:
        ss.ssvp_clip_median_depth(sess.ctx, 15)
    assert e2.value.code == ss.SSVP_ENOCLIP
    sess.load(15, tiny)
    sess.load(16, tiny)
    np.testing.assert_array_equal(sess.run(15, 8, k=5, half_window=2).rgb, sess.run(16, 8, k=5, half_window=2).rgb)


def test_empty_frame_range_is_a_no_op(sess, tiny):
    """frame_begin == frame_end: nothing is gathered, the output and the statistics stay as they are."""
    ss = sess.ss
    sess.load(0, tiny)
    before = sess.run(0, 4, k=5, half_window=2).rgb
    ss.ssvp_gather_filter(sess.ctx, sess.params(k=5, half_window=2, frame_begin=4, frame_end=4), [0])
    ss.ssvp_sync(sess.ctx)
    assert ss.ssvp_read_stats(sess.ctx) == (0, 0, 0.0)
    t = sess.torch
    out = t.empty((1, tiny.H, tiny.W, 3), dtype=t.float32, device=sess.dev)
    ss.ssvp_read_output(sess.ctx, 0, 4, 5, out)
    ss.ssvp_sync(sess.ctx)
    np.testing.assert_array_equal(out.cpu().numpy()[0], before)


def test_one_pixel_clip(sess):
    """A 1 x 1 clip: every window is the image border; the pixel keeps only its own sample."""
    c = synth.make_clip("planes3", 1, 1, 4, seed=3)
    sess.load(11, c)
    for O in range(c.F):
        g, o = _both(sess, c, 11, O, k=3, T=2)
        compare(g, o, 3)
        np.testing.assert_array_equal(g.rgb, c.rgb[O])


def test_window_beyond_the_clip_equals_the_clipped_window(sess, tiny):
    """T = 127 on a 16-frame clip gathers the same frames, in the same order, as T = 8 at O = 8."""
    sess.load(0, tiny)
    a = sess.run(0, 8, k=5, half_window=8).rgb
    b = sess.run(0, 8, k=5, half_window=127).rgb
    np.testing.assert_array_equal(a, b)


def test_launch_stats_match_oracle(sess, tiny):
    sess.load(0, tiny)
    g, o = _both(sess, tiny, 0, 8, k=5, T=15)
    e, a, w = sess.ss.ssvp_read_stats(sess.ctx)
    assert e == int(g.nexam.sum()) and a == int(g.nacc.sum())
    assert e == int(o.nexam.sum())
    assert abs(a - int(o.nacc.sum())) <= int(((o.codes & oracle.CODE_BAND) != 0).sum())
    assert w == pytest.approx(float(o.sumw.sum()), rel=1e-3)


def test_argument_errors(sess, tiny):
    ss = sess.ss
    sess.load(0, tiny)
    with pytest.raises(ss.SsvpError) as e:
        sess.run(0, 4, k=4)
    assert e.value.code == ss.SSVP_EINVAL
    with pytest.raises(ss.SsvpError) as e:
        sess.run(0, 4, crop=(150, 0, 20, 10))
    assert e.value.code == ss.SSVP_EINVAL
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_gather_filter(sess.ctx, sess.params(), [40])
    assert e.value.code == ss.SSVP_ENOCLIP
    import torch
    z = torch.zeros((2, 4, 4, 3), device="cuda")
    ss.ssvp_load_clip(sess.ctx, 9, 4, 4, 2, z, z[..., 0].contiguous())
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_gather_filter(sess.ctx, sess.params(), [9])
    assert e.value.code == ss.SSVP_ENOCAM
    K = np.array([[1.0, 0.1, 2], [0, 1, 2], [0, 0, 1]])
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_set_cameras(sess.ctx, 9, K, 0, np.tile(np.eye(3, 4), (2, 1, 1)))
    assert e.value.code == ss.SSVP_EINVAL


def test_buffers_in_the_wrong_memory_are_refused(sess, tiny):
    """Every buffer is checked for where it lives before any work touches it: host memory given as
    device memory (which a kernel would fault on), device memory given as host memory, and debug
    or output buffers that are not device memory are SSVP_EINVAL, and the context goes on working."""
    ss, t = sess.ss, sess.torch
    sess.load(0, tiny)
    want = sess.run(0, 4, k=5, half_window=2).rgb
    W, H, F = tiny.W, tiny.H, tiny.F
    rgb_d = t.from_numpy(tiny.rgb).to(sess.dev)
    dep_d = t.from_numpy(tiny.depth).to(sess.dev)
    cases = [
        lambda: ss.ssvp_load_clip(sess.ctx, 17, W, H, F, tiny.rgb, tiny.depth, ss.SSVP_MEM_DEVICE),
        lambda: ss.ssvp_load_clip(sess.ctx, 17, W, H, F, rgb_d, dep_d, ss.SSVP_MEM_HOST),
        lambda: ss.ssvp_load_clip(sess.ctx, 17, W, H, F, rgb_d, tiny.depth, ss.SSVP_MEM_DEVICE),
        lambda: ss.ssvp_read_output(sess.ctx, 0, 4, 5, np.zeros((1, H, W, 3), np.float32), ss.SSVP_MEM_DEVICE),
        lambda: ss.ssvp_read_output(sess.ctx, 0, 4, 5, t.zeros((1, H, W, 3), device=sess.dev), ss.SSVP_MEM_HOST),
        lambda: ss.ssvp_superres(sess.ctx, sess.params(gather=ss.SSVP_GATHER_FRUSTUM, frame_begin=4, frame_end=5), 0,
                                 2, np.zeros((1, 2 * H, 2 * W, 3), np.float32).ctypes.data),
    ]
    host_rec = np.zeros((H, W, 5, 4), np.int32)
    p = sess.params(k=5, half_window=2, frame_begin=4, frame_end=5)
    p.membership_out = host_rec.ctypes.data
    cases.append(lambda: ss.ssvp_gather_filter(sess.ctx, p, [0]))
    for call in cases:
        with pytest.raises(ss.SsvpError) as e:
            call()
        assert e.value.code == ss.SSVP_EINVAL and "memory" in str(e.value)
    assert not host_rec.any()
    # arguments the library reads or writes on the host, given device addresses through the C ABI
    import ctypes
    lib = ss.lib
    k_d = t.from_numpy(np.ascontiguousarray(tiny.K, np.float64)).to(sess.dev)
    w_d = t.from_numpy(np.ascontiguousarray(tiny.w2c, np.float64)).to(sess.dev)
    f_d = t.zeros(64, dtype=t.float64, device=sess.dev)
    for rc in (lib.ssvp_set_cameras(sess.ctx, 0, k_d.data_ptr(), 1, w_d.data_ptr()),
               lib.ssvp_set_shutter(sess.ctx, ctypes.cast(f_d.data_ptr(), ctypes.POINTER(ctypes.c_float)), 2),
               lib.ssvp_frame_sharpness(sess.ctx, 0, ctypes.cast(f_d.data_ptr(), ctypes.POINTER(ctypes.c_double))),
               lib.ssvp_clip_median_depth(sess.ctx, 0, ctypes.cast(f_d.data_ptr(), ctypes.POINTER(ctypes.c_float)))):
        assert rc == ss.SSVP_EINVAL and "memory" in ss.ssvp_last_error(sess.ctx)
    np.testing.assert_array_equal(sess.run(0, 4, k=5, half_window=2).rgb, want)


def test_full_size_sampled_against_oracle(sess):
    """1920x1080, +-30 frames, k = 7 in the benchmark's launch (all pixels of the output frame,
    no debug outputs); sampled crops compared with the oracle."""
    clip = synth.make_clip("room", 1920, 1080, 61, seed=0)
    sess.load(10, clip, colour_fmt=0)
    O = 30
    g = sess.run(10, O, k=7, half_window=30)
    med = oracle.median_depth(clip.depth)
    prm = oracle_params(med, 7, 30)
    v = oracle.ClipView.of(clip)
    worst = []
    for crop in [(0, 0, 24, 24), (960, 540, 24, 24), (1896, 1056, 24, 24), (400, 900, 24, 24)]:
        x0, y0, cw, ch = crop
        o = oracle.gather_filter(v, prm, O, crop=crop, membership=True)
        band = ((o.codes & oracle.CODE_BAND) != 0).any(axis=(-1, -2, -3)) | ((o.amb == 1) & (o.status == 1)).any(-1)
        err = np.abs(g.rgb[y0:y0 + ch, x0:x0 + cw] - o.rgb).max(-1)
        assert err[~band].max() <= COLOUR_TOL
        worst.append(err[~band].max())
    e, a, w = sess.ss.ssvp_read_stats(sess.ctx)
    assert a >= clip.W * clip.H  # every valid pixel accepts at least its own sample


def test_queued_reload_is_ordered_with_the_work_around_it(sess, tiny):
    """A clip load runs on the context's internal load stream: it must start only after the work
    queued before it (a gather of the old contents and an asynchronous read of its output) and
    finish before the work queued after it (a gather of the new contents), with no
    synchronisation between the calls."""
    t, ss = sess.torch, sess.ss
    other = synth.make_clip("room", tiny.W, tiny.H, tiny.F, seed=9)
    sess.load(12, tiny)
    want_old = sess.run(12, 8, k=5, half_window=15).rgb
    sess.load(13, other)
    want_new = sess.run(13, 8, k=5, half_window=15).rgb
    p = sess.params(k=5, half_window=15, frame_begin=8, frame_end=9)
    a = t.empty((1, tiny.H, tiny.W, 3), dtype=t.float32, device=sess.dev)
    b = t.empty_like(a)
    rgb_h = t.from_numpy(other.rgb).pin_memory()
    dep_h = t.from_numpy(other.depth).pin_memory()
    for rep in range(2):
        ss.ssvp_gather_filter(sess.ctx, p, [12])
        ss.ssvp_read_output(sess.ctx, 12, 8, 9, a)  # device copy: queued, not waited for
        ss.ssvp_load_clip(sess.ctx, 12, tiny.W, tiny.H, tiny.F, rgb_h, dep_h, ss.SSVP_MEM_HOST, 0)
        ss.ssvp_set_cameras(sess.ctx, 12, other.K, 1, other.w2c)
        ss.ssvp_gather_filter(sess.ctx, p, [12])
        ss.ssvp_read_output(sess.ctx, 12, 8, 9, b)
        ss.ssvp_sync(sess.ctx)
        np.testing.assert_array_equal(a.cpu().numpy()[0], want_old if rep == 0 else want_new)
        np.testing.assert_array_equal(b.cpu().numpy()[0], want_new)
