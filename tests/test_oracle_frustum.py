"""Pins of the oracle's frustum gather (Sec. "Sample Gathering", Eq. 1-2) against closed forms.

The frustum of pixel p is the square of side l around it swept over O depths (near, far); a
pixel q of frame J is a sample when its back-projection lands in it, |p - p'|_1 < l / 2
(Eq. 2 as printed).  Closed forms used here:
  * a camera moving exactly one pixel footprint per frame over a fronto-parallel plane sees the
    scene point of (u, v) of O at (u - (J - O), v) of J, so S(p) in J is the L1 ball of radius
    < l / 2 around that pixel (5 pixels for l = 3, 1 for l = 1, 13 for l = 5);
  * in J = O the back-projection is the identity, so S(p) from O is the L1 ball around p itself;
  * a rigid motion of the world and all cameras changes nothing;
  * a larger l never loses a sample;
  * an independent scan in numpy through world coordinates (c2w of J, then w2c and K of O)
    accepts the same pixels, with a near and far plane that cut the scene.
"""
import numpy as np
import pytest

import oracle
import synth


def _frustum_params(c, T, l=3.0, mode=oracle.MODE_MEAN, **kw):
    p = oracle.default_params(c.depth, mode=mode, k=1, T=T, **kw)
    p.gather, p.frustum_l = oracle.GATHER_FRUSTUM, l
    return p


def _ball(l):
    h = int(np.ceil(l / 2))
    return [(dx, dy) for dy in range(-h, h + 1) for dx in range(-h, h + 1) if abs(dx) + abs(dy) < l / 2]


@pytest.mark.parametrize("l,n_ball", [(1.0, 1), (3.0, 5), (5.0, 13)])
def test_exact_shift_frustum_sets_are_l1_balls(l, n_ball):
    c = synth.make_clip("exact_shift", 40, 24, 7, seed=1)
    v = oracle.ClipView.of(c)
    O, T = 3, 3
    p = _frustum_params(c, T, l)
    ball = _ball(l)
    assert len(ball) == n_ball
    r = oracle.frustum_filter(v, p, O, membership=True)
    H, W = c.H, c.W
    want_sum = np.zeros((H, W, 3))
    want_n = np.zeros((H, W), np.int64)
    for j in range(2 * T + 1):
        J = O - T + j
        cnt = np.zeros((H, W), np.int32)
        for vv in range(H):
            for uu in range(W):
                for dx, dy in ball:
                    qx, qy = uu - (J - O) + dx, vv + dy
                    if 0 <= qx < W and 0 <= qy < H:
                        cnt[vv, uu] += 1
                        want_sum[vv, uu] += c.rgb[J, qy, qx]
        np.testing.assert_array_equal(r.count[:, :, j], cnt)
        want_n += cnt
    assert not r.band.any()
    np.testing.assert_array_equal(r.nacc, want_n)
    # mode "mean": the plain average of exactly those input colours
    np.testing.assert_allclose(r.rgb, want_sum / want_n[..., None], atol=1e-12, rtol=0)
    # the per-frame accept maps of a few pixels are the shifted balls themselves
    for (uu, vv, J) in [(0, 0, 0), (20, 11, 5), (39, 23, 6), (5, 12, 3)]:
        m = oracle.bruteforce(v, p, O, uu, vv, J)
        want = np.zeros_like(m)
        for dx, dy in ball:
            qx, qy = uu - (J - O) + dx, vv + dy
            if 0 <= qx < W and 0 <= qy < H:
                want[qy, qx] = 1
        np.testing.assert_array_equal(m, want)


def test_self_frame_set_is_the_l1_ball_around_p():
    """T = 0 on a generic scene: G_{O<-O} is exact, so S(p) is p and its 4-neighbours (l = 3)
    with valid depth, whatever their depths; l = 1 returns I(p) itself."""
    c = synth.make_clip("room", 48, 27, 3, seed=5)
    c.depth[1, 4:9, 10:20] = np.nan  # invalid samples are never gathered
    v = oracle.ClipView.of(c)
    O, H, W = 1, c.H, c.W
    r = oracle.frustum_filter(v, _frustum_params(c, 0, 3.0), O, membership=True)
    valid = np.isfinite(c.depth[O]) & (c.depth[O] > 0)
    want_n = np.zeros((H, W), np.int64)
    want_sum = np.zeros((H, W, 3))
    for dx, dy in _ball(3.0):
        sh_valid = np.zeros((H, W), bool)
        sh_rgb = np.zeros((H, W, 3))
        ys, yd = slice(max(dy, 0), H + min(dy, 0)), slice(max(-dy, 0), H + min(-dy, 0))
        xs, xd = slice(max(dx, 0), W + min(dx, 0)), slice(max(-dx, 0), W + min(-dx, 0))
        sh_valid[yd, xd] = valid[ys, xs]
        sh_rgb[yd, xd] = c.rgb[O][ys, xs]
        want_n += sh_valid
        want_sum += sh_rgb * sh_valid[..., None]
    want_n[~valid] = 0  # an invalid reference depth gives c_ref and no samples
    np.testing.assert_array_equal(r.nacc, want_n)
    ok = valid & (want_n > 0)
    np.testing.assert_allclose(r.rgb[ok], (want_sum / np.maximum(want_n, 1)[..., None])[ok], atol=1e-12, rtol=0)
    np.testing.assert_array_equal(r.rgb[~valid], c.rgb[O][~valid])
    r1 = oracle.frustum_filter(v, _frustum_params(c, 0, 1.0), O)
    np.testing.assert_array_equal(r1.rgb[valid], c.rgb[O][valid].astype(np.float64))


def test_rigid_world_motion_changes_nothing():
    c = synth.make_clip("room", 40, 24, 7, seed=2)
    v = oracle.ClipView.of(c)
    p = _frustum_params(c, 3, 3.0, mode=oracle.MODE_DENOISE, sigma_xyz=0.2)
    r = oracle.frustum_filter(v, p, 3, membership=True)
    # world' = R x + t: w2c' = w2c [R^T | -R^T t]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]]) @ \
        np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    t = np.array([3.0, -1.0, 2.0])
    w2c = np.empty_like(c.w2c)
    for f in range(c.F):
        Rf, tf = c.w2c[f, :, :3], c.w2c[f, :, 3]
        w2c[f, :, :3] = Rf @ R.T
        w2c[f, :, 3] = tf - Rf @ R.T @ t
    r2 = oracle.frustum_filter(oracle.ClipView(c.rgb, c.depth, c.K, w2c), p, 3, membership=True)
    ok = (r.band == 0).all(axis=-1) & (r2.band == 0).all(axis=-1)
    assert ok.mean() > 0.9
    np.testing.assert_array_equal(r.count[ok], r2.count[ok])
    np.testing.assert_array_equal(r.hash[ok], r2.hash[ok])
    np.testing.assert_allclose(r.rgb[ok], r2.rgb[ok], atol=1e-9, rtol=0)


def test_larger_frustum_never_loses_a_sample():
    c = synth.make_clip("room", 40, 24, 7, seed=3)
    v = oracle.ClipView.of(c)
    prev = None
    for l in (1.0, 2.0, 3.0, 5.0):
        p = _frustum_params(c, 3, l)
        maps = np.stack([oracle.bruteforce(v, p, 3, u, w, J) for (u, w) in [(7, 5), (30, 18)] for J in (0, 3, 6)])
        if prev is not None:
            assert (maps >= prev).all()
            assert maps.sum() > prev.sum()
        prev = maps


def _world_route_map(c, O, u, v, J, l, near, far):
    """Every pixel of J tested through world coordinates: X_w = c2w_J (d K_J^-1 q), X_O = w2c_O X_w."""
    H, W = c.H, c.W
    qy, qx = np.mgrid[0:H, 0:W].astype(np.float64)
    d = c.depth[J].astype(np.float64)
    rays = np.stack([qx, qy, np.ones_like(qx)], -1) @ np.linalg.inv(c.K[J]).T
    Xc = rays * d[..., None]
    RJ, tJ = c.w2c[J, :, :3], c.w2c[J, :, 3]
    Xw = (Xc - tJ) @ RJ  # R^T (x - t), row vectors
    RO, tO = c.w2c[O, :, :3], c.w2c[O, :, 3]
    XO = Xw @ RO.T + tO
    z = XO[..., 2]
    with np.errstate(invalid="ignore", divide="ignore"):
        pix = XO @ c.K[O].T
        up, vp = pix[..., 0] / z, pix[..., 1] / z
        l1 = np.abs(u - up) + np.abs(v - vp)
        ok = np.isfinite(d) & (d > 0) & (z > near) & (z < far) & (l1 < l / 2)
        band = np.abs(l1 - l / 2) < 1e-6
    return ok.astype(np.uint8), band


def test_matches_a_scan_through_world_coordinates_with_near_and_far_planes():
    c = synth.make_clip("room", 48, 27, 9, seed=4)
    med = oracle.median_depth(c.depth)
    v = oracle.ClipView.of(c)
    for near, far in [(0.01, 1000.0), (0.8 * med, 1.3 * med)]:
        p = _frustum_params(c, 4, 3.0, near_plane=near, far_plane=far)
        n_total = 0
        for (u, w) in [(3, 2), (24, 13), (45, 25), (10, 20)]:
            for J in (0, 2, 4, 6, 8):
                got = oracle.bruteforce(v, p, 4, u, w, J)
                want, band = _world_route_map(c, 4, u, w, J, 3.0, near, far)
                diff = (got != want) & ~band
                assert not diff.any(), (near, far, u, w, J, np.argwhere(diff)[:5])
                n_total += int(got.sum())
        assert n_total > 20
