"""Batched plans (persistent launch of uneven clips, CUDA graph, autotuner) against the plain path."""
import numpy as np
import pytest

import synth
from _gpu import Session

pytestmark = pytest.mark.gpu

SIZES = [("planes3", 77, 45, 6, 1), ("room", 96, 54, 9, 2), ("planes3", 160, 90, 16, 3)]


@pytest.fixture(scope="module")
def sess():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    s = Session()
    for i, (preset, W, H, F, seed) in enumerate(SIZES):
        s.load(30 + i, synth.make_clip(preset, W, H, F, seed=seed), colour_fmt=1)
    yield s
    s.close()


def _outputs(sess):
    t = sess.torch
    outs = []
    for i, (_, W, H, F, _) in enumerate(SIZES):
        o = t.empty((F, H, W, 3), dtype=t.float32, device=sess.dev)
        sess.ss.ssvp_read_output(sess.ctx, 30 + i, 0, F, o)
        outs.append(o)
    sess.ss.ssvp_sync(sess.ctx)
    return [o.cpu().numpy() for o in outs]


def _plain(sess, p):
    totals = np.zeros(3)
    for i in range(len(SIZES)):
        sess.ss.ssvp_gather_filter(sess.ctx, p, [30 + i])
        totals += np.array(sess.ss.ssvp_read_stats(sess.ctx))
    return _outputs(sess), totals


def test_default_plan_matches_the_plain_path(sess):
    """Same tiles as the plain launch: the same samples with the same weights (identical counts),
    summed in the same order (two at a time in packed partial sums in both kernels), so colours
    agree to the bit; graph replays are bitwise identical."""
    ss = sess.ss
    p = sess.params(k=5, half_window=3)
    want, totals = _plain(sess, p)
    plan = ss.ssvp_plan_create(sess.ctx, p, [30, 31, 32])
    try:
        cfg, n_items, grid = ss.ssvp_plan_get_config(plan)
        assert (cfg.tile_rows, cfg.frame_chunk) == (8, 1) and grid > 0
        assert n_items == sum(((W + 31) // 32) * ((H + 7) // 8) * F for _, W, H, F, _ in SIZES)
        first = None
        for rep in range(2):
            ss.ssvp_plan_launch(plan)
            got = _outputs(sess)
            for a, b in zip(got, want):
                np.testing.assert_array_equal(a, b)
            if first is None:
                first = [g.copy() for g in got]
            else:
                for a, b in zip(got, first):
                    np.testing.assert_array_equal(a, b)
            e, acc, w = ss.ssvp_read_stats(sess.ctx)
            assert (e, acc) == (totals[0], totals[1])
            assert w == pytest.approx(totals[2], rel=1e-6)
    finally:
        ss.ssvp_plan_destroy(plan)


@pytest.mark.parametrize("rows,chunk", [(4, 1), (4, 4), (8, 3)])
def test_other_shapes_agree_with_the_plain_path(sess, rows, chunk):
    ss = sess.ss
    p = sess.params(k=7, half_window=4)
    want, totals = _plain(sess, p)
    plan = ss.ssvp_plan_create(sess.ctx, p, [30, 31, 32], ss.ssvp_plan_config(rows, chunk))
    try:
        ss.ssvp_plan_launch(plan)
        got = _outputs(sess)
        e, acc, _ = ss.ssvp_read_stats(sess.ctx)
    finally:
        ss.ssvp_plan_destroy(plan)
    # a different tile base changes the double-float rounding of the reference point at the
    # 1e-12 level: only candidates on the radius can flip
    diff = np.concatenate([np.abs(a - b).max(-1).ravel() for a, b in zip(got, want)])
    assert (diff > 1e-3).mean() < 1e-3
    assert abs(acc - totals[1]) <= 1e-5 * totals[1] + 5
    assert abs(e - totals[0]) <= 1e-4 * totals[0]


def test_autotune_and_reload_guard(sess):
    ss = sess.ss
    p = sess.params(k=7, half_window=4)
    best = ss.ssvp_autotune(sess.ctx, p, [30, 31, 32])
    assert best.tile_rows in (4, 8) and best.frame_chunk in (1, 2, 4, 8)
    plan = ss.ssvp_plan_create(sess.ctx, p, [30, 31, 32])
    try:
        cfg, _, _ = ss.ssvp_plan_get_config(plan)
        assert (cfg.tile_rows, cfg.frame_chunk) == (best.tile_rows, best.frame_chunk)
        ss.ssvp_plan_launch(plan)
        ss.ssvp_sync(sess.ctx)
        sess.load(31, synth.make_clip("room", 96, 54, 9, seed=2), colour_fmt=1)
        with pytest.raises(ss.SsvpError) as e:
            ss.ssvp_plan_launch(plan)
        assert e.value.code == ss.SSVP_ENOCLIP
    finally:
        ss.ssvp_plan_destroy(plan)


def test_plan_argument_checks(sess):
    ss = sess.ss
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_plan_create(sess.ctx, sess.params(mode=1), [30])
    assert e.value.code == ss.SSVP_EINVAL
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_plan_create(sess.ctx, sess.params(), [30], ss.ssvp_plan_config(5, 1))
    assert e.value.code == ss.SSVP_EINVAL
    with pytest.raises(ss.SsvpError) as e:
        ss.ssvp_plan_create(sess.ctx, sess.params(crop_w=8, crop_h=8), [30])
    assert e.value.code == ss.SSVP_EINVAL


def test_plan_update_after_same_shape_reloads_and_new_cameras(sess):
    """ssvp_plan_update keeps the captured graph and recomposes the geometry: after a same-shape
    reload with new contents and cameras, and after ssvp_set_cameras, the plan again gives the
    plain path's output to the bit; a reload with another shape is refused."""
    ss = sess.ss
    p = sess.params(k=5, half_window=3)
    plan = ss.ssvp_plan_create(sess.ctx, p, [30, 31, 32], ss.ssvp_plan_config(8, 1))
    try:
        ss.ssvp_plan_launch(plan)
        other = synth.make_clip("room", 96, 54, 9, seed=7)  # clip 31's shape, other scene and path
        sess.load(31, other, colour_fmt=1)
        with pytest.raises(ss.SsvpError) as e:
            ss.ssvp_plan_launch(plan)
        assert e.value.code == ss.SSVP_ENOCLIP
        ss.ssvp_plan_update(plan)
        ss.ssvp_plan_launch(plan)
        got = _outputs(sess)
        want, _ = _plain(sess, p)
        for a, b in zip(got, want):
            np.testing.assert_array_equal(a, b)
        c0 = synth.make_clip(*SIZES[0][:4], seed=SIZES[0][4])
        ss.ssvp_set_cameras(sess.ctx, 30, c0.K, 1, c0.w2c_true)  # the exact cameras instead
        ss.ssvp_plan_update(plan)
        ss.ssvp_plan_launch(plan)
        got = _outputs(sess)
        want, _ = _plain(sess, p)
        for a, b in zip(got, want):
            np.testing.assert_array_equal(a, b)
        sess.load(32, synth.make_clip("planes3", 160, 90, 12, seed=3), colour_fmt=1)  # another F
        with pytest.raises(ss.SsvpError) as e:
            ss.ssvp_plan_update(plan)
        assert e.value.code == ss.SSVP_EINVAL
    finally:
        ss.ssvp_plan_destroy(plan)
        for i, (preset, W, H, F, seed) in enumerate(SIZES):  # the module's clips as they were
            sess.load(30 + i, synth.make_clip(preset, W, H, F, seed=seed), colour_fmt=1)
