"""Device memory over repeated use: contexts created and destroyed, clips loaded, reloaded with
other shapes, appended to and unloaded, window / staged / frustum / aperture gathers, batched
plans created and destroyed, the learned filter set and run.  After every cycle the device's free
memory must come back to what it was after the first cycle (the library frees all it allocates;
the first cycle also pays for one-time costs such as module loading)."""
import pytest

import synth

pytestmark = pytest.mark.gpu

SLACK = 64 << 20  # bytes: allocator granularity and driver bookkeeping


def _cycle(ss, t, dev, clips, W1, b1, W2, b2):
    stream = t.cuda.current_stream(dev)
    ctx = ss.ssvp_create(0, stream)
    try:
        for cid, c in enumerate(clips):
            ss.ssvp_load_clip(ctx, cid, c.W, c.H, c.F, c.rgb, c.depth, ss.SSVP_MEM_HOST, cid % 2)
            ss.ssvp_set_cameras(ctx, cid, c.K, 1, c.w2c)
        p = ss.ssvp_params_default()
        p.k, p.half_window, p.frame_begin, p.frame_end = 5, 3, 1, 3
        for gather in (ss.SSVP_GATHER_WINDOW, ss.SSVP_GATHER_WINDOW_TMA):
            p.gather = gather
            ss.ssvp_gather_filter(ctx, p, [0, 1])
        p.gather, p.frustum_l = ss.SSVP_GATHER_FRUSTUM, 3.0
        ss.ssvp_gather_filter(ctx, p, [2])
        p.gather, p.mode, p.cap, p.lens_samples, p.aperture = ss.SSVP_GATHER_WINDOW, ss.SSVP_MODE_APERTURE, 9, 8, 0.05
        ss.ssvp_gather_filter(ctx, p, [0])
        p = ss.ssvp_params_default()
        p.k, p.half_window, p.frame_begin, p.frame_end = 5, 2, 0, -1
        plan = ss.ssvp_plan_create(ctx, p, [0, 2])  # both FP32 clips
        ss.ssvp_plan_launch(plan)
        ss.ssvp_plan_destroy(plan)
        ss.ssvp_set_mlp(ctx, W1, b1, W2, b2)
        p.mode, p.frame_begin, p.frame_end = ss.SSVP_MODE_LEARNED, 2, 3
        ss.ssvp_gather_filter(ctx, p, [0])
        c = clips[0]
        ss.ssvp_append_frames(ctx, 0, 2, c.rgb[:2], c.depth[:2], c.K[:2], 1, c.w2c[:2], ss.SSVP_MEM_HOST)
        # a reload of an id with another shape frees and reallocates its planes
        d = clips[1]
        ss.ssvp_load_clip(ctx, 0, d.W, d.H, d.F, d.rgb, d.depth, ss.SSVP_MEM_HOST, 0)
        ss.ssvp_sync(ctx)
        for cid in range(len(clips)):
            ss.ssvp_unload_clip(ctx, cid)
    finally:
        ss.ssvp_destroy(ctx)
    t.cuda.synchronize()


def test_repeated_use_frees_what_it_allocates():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import oracle
    import paper_2102_03011_gb300 as ss
    dev = torch.device("cuda:0")
    clips = [synth.make_clip("room", 96, 54, 8, seed=1), synth.make_clip("planes3", 80, 45, 6, seed=2),
             synth.make_clip("room", 64, 36, 7, seed=3)]
    W1, b1, W2, b2 = oracle.he_init(3)
    _cycle(ss, torch, dev, clips, W1, b1, W2, b2)
    torch.cuda.empty_cache()
    base = torch.cuda.mem_get_info(dev)[0]
    for _ in range(4):
        _cycle(ss, torch, dev, clips, W1, b1, W2, b2)
        torch.cuda.empty_cache()
        free = torch.cuda.mem_get_info(dev)[0]
        assert free >= base - SLACK, (base - free) / 2**20
