"""Kernel timing through the C ABI (ssvp_trace_enable / ssvp_trace_read): each traced call is
recorded under its kind with the right launch count, the times agree with CUDA events taken
around the same calls, reading clears the record, and nothing is recorded while tracing is off."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import Session

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
def clip():
    return synth.make_clip("room", 320, 180, 15, seed=4)


def _timed(sess, fn):
    t = sess.torch
    a, b = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
    t.cuda.synchronize()
    a.record(sess.stream)
    fn()
    b.record(sess.stream)
    t.cuda.synchronize()
    return a.elapsed_time(b)


def test_load_and_gathers_are_recorded_by_kind(sess, clip):
    ss = sess.ss
    ss.ssvp_trace_enable(sess.ctx, True)
    try:
        assert ss.ssvp_trace_read(sess.ctx) == {}
        sess.load(0, clip)
        rec = ss.ssvp_trace_read(sess.ctx)
        assert set(rec) == {"load"} and rec["load"][0] == 1 and rec["load"][1] > 0.0
        p = sess.params(half_window=7, frame_begin=7, frame_end=10)
        ext = _timed(sess, lambda: ss.ssvp_gather_filter(sess.ctx, p, [0]))
        rec = ss.ssvp_trace_read(sess.ctx)
        assert set(rec) == {"gather"} and rec["gather"][0] == 1  # one launch for the three frames
        assert 0.5 * ext <= rec["gather"][1] <= ext * 1.05 + 0.02
        assert ss.ssvp_trace_read(sess.ctx) == {}  # the read cleared the record
        pa = sess.params(mode=ss.SSVP_MODE_APERTURE, half_window=7, frame_begin=7, frame_end=8, aperture=0.05,
                         focal_depth=0.0, cap=31)
        ss.ssvp_gather_filter(sess.ctx, pa, [0])
        pf = sess.params(gather=ss.SSVP_GATHER_FRUSTUM, half_window=3, frame_begin=7, frame_end=8,
                         crop_x=100, crop_y=60, crop_w=40, crop_h=30)
        ss.ssvp_gather_filter(sess.ctx, pf, [0])
        ss.ssvp_gather_filter(sess.ctx, pf, [0])
        ss.ssvp_gather_filter(sess.ctx, p, [0])
        rec = ss.ssvp_trace_read(sess.ctx)
        # the frames' depth ranges are computed once, at the first frustum gather after the load
        assert {k: v[0] for k, v in rec.items()} == {"gather": 1, "aperture": 1, "frustum": 2, "load": 1}
        assert all(v[1] > 0.0 for v in rec.values())
        db = sess.params(mode=ss.SSVP_MODE_DEBLUR, half_window=7, frame_begin=7, frame_end=8)
        ss.ssvp_gather_filter(sess.ctx, db, [0])
        ss.ssvp_gather_filter(sess.ctx, db, [0])
        rec = ss.ssvp_trace_read(sess.ctx)
        assert {k: v[0] for k, v in rec.items()} == {"gather": 2, "load": 1}  # the Eq. 5 sums, once
    finally:
        ss.ssvp_trace_enable(sess.ctx, False)


def test_learned_filter_records_extraction_and_inference_per_frame(sess, clip):
    ss = sess.ss
    sess.load(1, clip)
    W1, b1, W2, b2 = oracle.he_init(5)
    ss.ssvp_set_mlp(sess.ctx, W1, b1, W2, np.array([0.2, 1.5]))
    p = sess.params(mode=ss.SSVP_MODE_LEARNED, half_window=5, frame_begin=6, frame_end=8)
    ss.ssvp_trace_enable(sess.ctx, True)
    try:
        ext = _timed(sess, lambda: ss.ssvp_gather_filter(sess.ctx, p, [1]))
        rec = ss.ssvp_trace_read(sess.ctx)
        assert {k: v[0] for k, v in rec.items()} == {"extract": 2, "infer": 2}
        assert rec["extract"][1] + rec["infer"][1] <= ext * 1.05 + 0.05
        c = sess.torch.from_numpy(clip.clean).to(sess.dev)
        cfg = ss.ssvp_train_config(steps=3, batch_pixels=512, lr=1e-3, bce_weight=0.1, seed=0, init=0)
        ss.ssvp_train(sess.ctx, p, [1], [c], cfg)
        rec = ss.ssvp_trace_read(sess.ctx)
        assert {k: v[0] for k, v in rec.items()} == {"extract": 3, "train": 3, "adam": 3}
    finally:
        ss.ssvp_trace_enable(sess.ctx, False)


def test_plan_launch_is_one_batch_entry_and_nothing_is_recorded_when_off(sess, clip):
    ss = sess.ss
    sess.load(2, clip)
    p = sess.params(half_window=5)
    plan = ss.ssvp_plan_create(sess.ctx, p, [2])
    try:
        ss.ssvp_trace_enable(sess.ctx, True)
        ss.ssvp_plan_launch(plan)
        ss.ssvp_plan_launch(plan)
        rec = ss.ssvp_trace_read(sess.ctx)
        assert set(rec) == {"batch"} and rec["batch"][0] == 2
        ss.ssvp_trace_enable(sess.ctx, False)
        ss.ssvp_plan_launch(plan)
        ss.ssvp_gather_filter(sess.ctx, sess.params(half_window=5, frame_begin=5, frame_end=6), [2])
        assert ss.ssvp_trace_read(sess.ctx) == {}
    finally:
        ss.ssvp_trace_enable(sess.ctx, False)
        ss.ssvp_plan_destroy(plan)
