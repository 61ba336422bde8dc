"""Seeded random parity cases of the gathers against the FP64 oracle: clip shapes from one pixel
up, windows reaching past the clip's ends, odd crops, radii from tight to loose, invalid depths,
both colour formats, the denoise and mean modes and both window gathers (global loads and
TMA-staged boxes); the virtual-aperture and frustum gathers with random caps, lens radii, focal
depths, frustum sizes and near / far planes; the learned weighting with random networks,
confidence thresholds and set sizes; super-resolution, inpainting and semi-transparency with random
scales, painted masks and crops; batched plans over random sets of uneven clips.  Every case must pass the same membership and colour comparison as the fixed
parity tests; the draws are fixed by the seed, so a failure names a reproducible case."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import (Session, compare, compare_aperture, compare_flagged, compare_frustum, oracle_params, run_frustum,
                  run_superres, superres_ref_valid)

pytestmark = pytest.mark.gpu

N_CASES = 32


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


def _case(i):
    rng = np.random.default_rng(9000 + i)
    W, H = int(rng.integers(1, 90)), int(rng.integers(1, 60))
    F = int(rng.integers(1, 9))
    k = int(rng.choice([1, 3, 5, 7, 9, 11]))
    return dict(
        preset=str(rng.choice(["planes3", "room"])), W=W, H=H, F=F, seed=int(rng.integers(0, 1000)), k=k,
        T=int(rng.integers(0, F + 3)), O=int(rng.integers(0, F)),
        x0=int(rng.integers(0, max(1, W // 2))), y0=int(rng.integers(0, max(1, H // 2))),
        radius_rel=float(rng.choice([0.002, 0.005, 0.02, 0.05])),
        mode=int(rng.choice([oracle.MODE_DENOISE, oracle.MODE_MEAN])), cfmt=int(rng.integers(0, 2)),
        bad_frac=float(rng.choice([0.0, 0.0, 0.1])), staged=bool(k <= 7 and rng.integers(0, 2)),
        bad_seed=int(rng.integers(0, 1 << 30)), cw_frac=0.3 + 0.7 * float(rng.random()),
        ch_frac=0.3 + 0.7 * float(rng.random()))


@pytest.mark.parametrize("i", range(N_CASES))
def test_random_case_matches_the_oracle(sess, i):
    c = _case(i)
    clip = synth.make_clip(c["preset"], c["W"], c["H"], c["F"], seed=c["seed"])
    depth = clip.depth.copy()
    if c["bad_frac"]:
        rng = np.random.default_rng(c["bad_seed"])
        bad = rng.random(depth.shape) < c["bad_frac"]
        depth[bad] = np.array([np.nan, 0.0, -1.0, np.inf], np.float32)[rng.integers(0, 4, int(bad.sum()))]
    rgb = clip.rgb if c["cfmt"] == 0 else clip.rgb.astype(np.float16).astype(np.float32)
    v = synth.Clip(clip.W, clip.H, clip.F, clip.K, clip.w2c, clip.w2c_true, rgb, depth, clip.clean, clip.depth_true)
    sess.load(30 + i % 8, v, colour_fmt=c["cfmt"])
    x0, y0 = c["x0"], c["y0"]
    cw = max(1, int(round((c["W"] - x0) * c["cw_frac"])))
    ch = max(1, int(round((c["H"] - y0) * c["ch_frac"])))
    crop = (x0, y0, cw, ch)
    ss = sess.ss
    g = sess.run(30 + i % 8, c["O"], crop=crop, membership=True, k=c["k"], half_window=c["T"], mode=c["mode"],
                 radius=-c["radius_rel"],
                 gather=ss.SSVP_GATHER_WINDOW_TMA if c["staged"] else ss.SSVP_GATHER_WINDOW)
    med = oracle.median_depth(depth)
    if not np.isfinite(med):
        # no valid depth anywhere: every pixel keeps its own colour
        np.testing.assert_array_equal(g.rgb, rgb[c["O"], y0:y0 + ch, x0:x0 + cw])
        return
    o = oracle.gather_filter(oracle.ClipView.of(v), oracle_params(med, c["k"], c["T"], mode=c["mode"],
                                                                  radius_rel=c["radius_rel"]),
                             c["O"], crop=crop, membership=True)
    compare(g, o, c["k"])


def _crop(c):
    x0, y0 = c["x0"], c["y0"]
    return (x0, y0, max(1, int(round((c["W"] - x0) * c["cw_frac"]))), max(1, int(round((c["H"] - y0) * c["ch_frac"]))))


def _clip(c):
    clip = synth.make_clip(c["preset"], c["W"], c["H"], c["F"], seed=c["seed"])
    depth = clip.depth.copy()
    if c["bad_frac"]:
        rng = np.random.default_rng(c["bad_seed"])
        bad = rng.random(depth.shape) < c["bad_frac"]
        depth[bad] = np.array([np.nan, 0.0, -1.0, np.inf], np.float32)[rng.integers(0, 4, int(bad.sum()))]
    return synth.Clip(clip.W, clip.H, clip.F, clip.K, clip.w2c, clip.w2c_true, clip.rgb, depth, clip.clean,
                      clip.depth_true)


@pytest.mark.parametrize("i", range(12))
def test_random_aperture_case_matches_the_oracle(sess, i):
    """The virtual-aperture gather (Eq. 13-14) on random shapes, caps, windows, lens radii and
    focal depths."""
    c = _case(100 + i)
    rng = np.random.default_rng(7000 + i)
    v = _clip(c)
    med = oracle.median_depth(v.depth)
    if not np.isfinite(med):
        return
    cap = int(rng.choice([1, 3, 9, 15, 31]))
    aperture = float(rng.choice([0.0, 0.02, 0.05, 0.1]))
    focal = float(med * rng.choice([0.5, 1.0, 2.0]))
    lens = int(rng.choice([1, 4, 16, 64]))
    sess.load(40 + i % 4, v)
    crop = _crop(c)
    g = sess.run(40 + i % 4, c["O"], crop=crop, membership=True, mode=1, k=c["k"], half_window=c["T"],
                 aperture=aperture, focal_depth=focal, cap=cap, lens_samples=lens)
    prm = oracle.Params(mode=oracle.MODE_APERTURE, k=c["k"], T=c["T"], aperture=aperture, focal_depth=focal,
                        lens_samples=lens, cap=cap)
    o = oracle.gather_filter(oracle.ClipView.of(v), prm, c["O"], crop=crop, membership=True)
    compare_aperture(g, o, cap)


@pytest.mark.parametrize("i", range(12))
def test_random_frustum_case_matches_the_oracle(sess, i):
    """The paper's frustum gather (Eq. 1-2) on random shapes, frustum sizes, windows and near /
    far planes, denoise and mean modes."""
    c = _case(200 + i)
    rng = np.random.default_rng(8000 + i)
    v = _clip(c)
    med = oracle.median_depth(v.depth)
    if not np.isfinite(med):
        return
    l = float(rng.choice([1.0, 2.5, 3.0, 5.0]))
    near, far = (0.01, 1000.0) if rng.integers(0, 2) else (0.6 * med, 1.5 * med)
    prm = oracle.Params(mode=c["mode"], k=1, T=c["T"], radius=0.005 * med, sigma_xyz=0.03 * med,
                        gather=oracle.GATHER_FRUSTUM, frustum_l=l, near_plane=near, far_plane=far)
    sess.load(44 + i % 4, v)
    crop = _crop(c)
    g = run_frustum(sess, 44 + i % 4, c["O"], crop=crop, membership=True, half_window=c["T"], mode=c["mode"],
                    frustum_l=l, sigma_xyz=prm.sigma_xyz, near_plane=near, far_plane=far)
    o = oracle.frustum_filter(oracle.ClipView.of(v), prm, c["O"], crop=crop, membership=True)
    x0, y0, cw, ch = crop
    d = v.depth[c["O"], y0:y0 + ch, x0:x0 + cw]
    compare_frustum(g, o, np.isfinite(d) & (d > 0))


@pytest.mark.parametrize("i", range(10))
def test_random_learned_case_matches_the_oracle(sess, i):
    """The learned weighting (capped sets, tcgen05 inference, plain fallback) on random shapes,
    windows, radii (up to sets past the 64-sample cap), networks and confidence thresholds, pixel
    by pixel against the oracle with the tensor cores' BF16 rounding."""
    rng = np.random.default_rng(6000 + i)
    W, H, F = int(rng.integers(8, 70)), int(rng.integers(4, 40)), int(rng.integers(2, 9))
    k, T, O = int(rng.choice([1, 3, 5, 7, 7])), int(rng.integers(1, F + 2)), int(rng.integers(0, F))
    radius_rel = float(rng.choice([0.005, 0.05, 0.1, 0.2]))
    tau = float(rng.choice([0.0, 0.5, 0.5, 2.0]))
    clip = synth.make_clip(str(rng.choice(["planes3", "room"])), W, H, F, seed=int(rng.integers(0, 1000)))
    x0, y0 = int(rng.integers(0, W // 2)), int(rng.integers(0, H // 2))
    crop = (x0, y0, max(1, int((W - x0) * (0.3 + 0.7 * rng.random()))), max(1, int((H - y0) * (0.3 + 0.7 * rng.random()))))
    W1, b1, W2, b2 = oracle.he_init(int(rng.integers(0, 1000)))
    b1 = rng.normal(0, 0.1, 64)
    b2 = np.array([rng.normal(0, 0.5), rng.normal(0.5, 1.0)])
    sess.load(50 + i % 4, clip)
    sess.ss.ssvp_set_mlp(sess.ctx, W1, b1, W2, b2)
    g = sess.run(50 + i % 4, O, crop=crop, mode=2, k=k, half_window=T, radius=-radius_rel, conf_threshold=tau)
    prm = oracle.default_params(clip.depth, k=k, T=T, radius_rel=radius_rel)
    of, oc, on, op = oracle.learned_crop(oracle.ClipView.of(clip), prm, O, crop=crop)
    o = oracle.gather_filter(oracle.ClipView.of(clip), prm, O, crop=crop, membership=True)
    flagged = ((o.codes & oracle.CODE_BAND) != 0).any(axis=(-1, -2, -3)) | ((o.amb == 1) & (o.status == 1)).any(-1)
    worst = 0.0
    for y in range(crop[3]):
        for x in range(crop[2]):
            if flagged[y, x]:
                continue
            _, ofin, conf, _ = oracle.mlp_pixel(of[y, x], oc[y, x], on[y, x], W1, b1, W2, b2, round_bf16=True,
                                                tau=tau, plain=op[y, x])
            if on[y, x] > 0 and abs(conf - tau) < 1e-3:
                continue  # the fallback decision is a tie between FP32 and FP64
            worst = max(worst, float(np.abs(g.rgb[y, x] - ofin).max()))
    assert worst <= 1e-3, worst


@pytest.mark.parametrize("i", range(8))
def test_random_superres_case_matches_the_oracle(sess, i):
    """Super-resolution (Eq. 6-7) on random shapes, scales 1-4, frustum sizes, windows and
    output-grid crops, with invalid depths in some cases."""
    rng = np.random.default_rng(5000 + i)
    W, H, F = int(rng.integers(6, 48)), int(rng.integers(4, 30)), int(rng.integers(1, 7))
    scale, l = int(rng.choice([1, 2, 3, 4])), float(rng.choice([1.0, 2.0, 3.0]))
    T, O = int(rng.integers(0, F + 1)), int(rng.integers(0, F))
    mode = int(rng.choice([oracle.MODE_DENOISE, oracle.MODE_MEAN]))
    c = dict(preset=str(rng.choice(["planes3", "room"])), W=W, H=H, F=F, seed=int(rng.integers(0, 1000)),
             bad_frac=float(rng.choice([0.0, 0.05])), bad_seed=int(rng.integers(0, 1 << 30)))
    v = _clip(c)
    med = oracle.median_depth(v.depth)
    if not np.isfinite(med):
        return
    Wo, Ho = W * scale, H * scale
    x0, y0 = int(rng.integers(0, Wo // 2 + 1)), int(rng.integers(0, Ho // 2 + 1))
    crop = (x0, y0, max(1, int((Wo - x0) * (0.3 + 0.7 * rng.random()))), max(1, int((Ho - y0) * (0.3 + 0.7 * rng.random()))))
    p = oracle.Params(mode=mode, k=1, T=T, radius=0.005 * med, sigma_rgb=50.0 / 255.0, sigma_xyz=0.03 * med,
                      gather=oracle.GATHER_FRUSTUM, frustum_l=l)
    sess.load(54 + i % 4, v)
    g = run_superres(sess, 54 + i % 4, O, scale, crop=crop, membership=True, half_window=T, mode=mode, frustum_l=l,
                     sigma_rgb=p.sigma_rgb, sigma_xyz=p.sigma_xyz)
    o = oracle.superres_filter(oracle.ClipView.of(v), p, O, scale, crop=crop, membership=True)
    compare_frustum(g, o, superres_ref_valid(v, O, scale, crop))


@pytest.mark.parametrize("i", range(8))
def test_random_inpaint_case_matches_the_oracle(sess, i):
    """Inpainting and semi-transparency (Eq. 8-9 and the variant after it) with random painted
    masks (discs drifting over the frames), windows, crops and Eq. 4 scales."""
    rng = np.random.default_rng(4000 + i)
    W, H, F = int(rng.integers(16, 64)), int(rng.integers(10, 40)), int(rng.integers(2, 8))
    T, O = int(rng.integers(1, F + 1)), int(rng.integers(0, F))
    semi = bool(rng.integers(0, 2))
    c = dict(preset=str(rng.choice(["planes3", "room"])), W=W, H=H, F=F, seed=int(rng.integers(0, 1000)),
             bad_frac=float(rng.choice([0.0, 0.05])), bad_seed=int(rng.integers(0, 1 << 30)))
    v = _clip(c)
    med = oracle.median_depth(v.depth)
    if not np.isfinite(med):
        return
    yy, xx = np.mgrid[0:H, 0:W]
    cx, cy, r = rng.uniform(0, W), rng.uniform(0, H), rng.uniform(2, max(3, min(W, H) / 2))
    vx, vy = rng.uniform(-2, 2), rng.uniform(-1, 1)
    mask = np.stack([((xx - cx - vx * f) ** 2 + (yy - cy - vy * f) ** 2 < r * r) for f in range(F)]).astype(np.uint8)
    # a crop around the disc as it lies in frame O (clipped to the image)
    ox, oy = cx + vx * O, cy + vy * O
    x0 = int(np.clip(ox - r - rng.integers(0, 4), 0, W - 1))
    y0 = int(np.clip(oy - r - rng.integers(0, 4), 0, H - 1))
    crop = (x0, y0, int(np.clip(2 * r + rng.integers(1, 8), 1, W - x0)), int(np.clip(2 * r + rng.integers(1, 8), 1, H - y0)))
    cid = 58 + i % 4
    sess.load(cid, v)
    sess.ss.ssvp_set_mask(sess.ctx, cid, mask)
    if semi:
        sx = float(med * rng.choice([0.01, 0.03, 0.1]))
        g = run_frustum(sess, cid, O, crop=crop, membership=True, half_window=T, mode=sess.ss.SSVP_MODE_SEMI,
                        sigma_rgb=80.0 / 255.0, sigma_xyz=sx)
        prm = oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=0.01, sigma_rgb=80.0 / 255.0, sigma_xyz=sx,
                            gather=oracle.GATHER_FRUSTUM, frustum_l=3.0)
    else:
        g = run_frustum(sess, cid, O, crop=crop, membership=True, half_window=T, mode=sess.ss.SSVP_MODE_INPAINT,
                        sigma_rgb=55.0 / 255.0)
        prm = oracle.Params(mode=oracle.MODE_DENOISE, k=1, T=T, radius=0.01, sigma_rgb=55.0 / 255.0,
                            gather=oracle.GATHER_FRUSTUM, frustum_l=3.0)
    o = oracle.inpaint_filter(oracle.ClipView.of(v), prm, mask, O, crop=crop, membership=True, semi=semi)
    x0, y0, cw, ch = crop
    compare_frustum(g, o, mask[O, y0:y0 + ch, x0:x0 + cw] != 0)


@pytest.mark.parametrize("i", range(6))
def test_random_batched_plan_matches_the_oracle(sess, i):
    """A graph-captured batched plan over 1-5 clips of random, uneven shapes and lengths (from one
    pixel and one frame up), with a random tile height and frame chunk, both colour formats and
    both modes: every output frame of every clip against the oracle."""
    ss, t = sess.ss, sess.torch
    rng = np.random.default_rng(3000 + i)
    n = int(rng.integers(1, 6))
    cfmt = int(rng.integers(0, 2))
    k, T = int(rng.choice([1, 3, 5, 7, 9])), int(rng.integers(0, 7))
    mode = int(rng.choice([oracle.MODE_DENOISE, oracle.MODE_MEAN]))
    clips, ids = [], []
    for j in range(n):
        W, H, F = int(rng.integers(1, 80)), int(rng.integers(1, 50)), int(rng.integers(1, 11))
        c = synth.make_clip(str(rng.choice(["planes3", "room"])), W, H, F, seed=int(rng.integers(0, 1000)))
        if cfmt:
            c = synth.Clip(c.W, c.H, c.F, c.K, c.w2c, c.w2c_true, c.rgb.astype(np.float16).astype(np.float32), c.depth,
                           c.clean, c.depth_true)
        sess.load(20 + j, c, colour_fmt=cfmt)
        clips.append(c)
        ids.append(20 + j)
    fb = int(rng.integers(0, min(c.F for c in clips)))
    cfg = ss.ssvp_plan_config()
    cfg.tile_rows, cfg.frame_chunk = int(rng.choice([4, 8])), int(rng.choice([1, 2, 3, 5, 16]))
    p = sess.params(k=k, half_window=T, frame_begin=fb, frame_end=-1, mode=mode)
    plan = ss.ssvp_plan_create(sess.ctx, p, ids, cfg)
    try:
        ss.ssvp_plan_launch(plan)
        ss.ssvp_sync(sess.ctx)
    finally:
        ss.ssvp_plan_destroy(plan)
    for cid, c in zip(ids, clips):
        out = t.empty((c.F, c.H, c.W, 3), dtype=t.float32, device=sess.dev)
        ss.ssvp_read_output(sess.ctx, cid, 0, c.F, out)
        ss.ssvp_sync(sess.ctx)
        out = out.cpu().numpy()
        med = oracle.median_depth(c.depth)
        if not np.isfinite(med):
            continue
        prm = oracle_params(med, k, T, mode=mode)
        for O in range(fb, c.F):
            o = oracle.gather_filter(oracle.ClipView.of(c), prm, O, membership=True)
            s = compare_flagged(out[O], o)
            assert s["differing"] <= 0.01 * s["pixels"] + 2, s
