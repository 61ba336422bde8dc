"""Pins of the oracle's virtual-aperture mode (Sec. "Virtual aperture", Eq. 13-14), no GPU.

On the optical axis of a camera translating exactly one pixel footprint per frame over a
fronto-parallel plane at depth Z, the cone is a circular cylinder section of radius
a(Z) = a0 + A |z0 - Z| / z0 around the axis, so the accepted set in every frame is a disc of
lattice points known in closed form, all weights are equal (same depth, same cone radius), and
the output is the plain mean of the clean colours in those discs.
"""
import numpy as np
import pytest

import oracle
import synth


def _axis_clip(F=7, seed=1):
    c = synth.make_clip("exact_shift", 65, 37, F, seed=seed)  # odd sizes: pixel (32, 18) is on the axis
    fx = c.K[0, 0, 0]
    assert c.K[0, 0, 2] == 32.0 and c.K[0, 1, 2] == 18.0
    return c, fx, float(c.depth[0, 0, 0])


@pytest.mark.parametrize("z0_rel,A", [(0.5, 0.05), (1.0, 0.05), (2.0, 0.03), (0.7, 0.0)])
def test_cone_on_axis_is_a_closed_form_disc(z0_rel, A):
    c, fx, Z = _axis_clip()
    z0 = z0_rel * Z
    O, T, u, v = 3, 3, 32, 18
    prm = oracle.Params(mode=oracle.MODE_APERTURE, k=7, T=T, aperture=A, focal_depth=z0, a0=0.3 * Z / fx,
                        lens_samples=16, cap=31)
    r = oracle.gather_filter(oracle.ClipView.of(c), prm, O, crop=(u, v, 1, 1), membership=True)
    a = prm.a0 + A * abs(z0 - Z) / z0
    step = 1.0 / 32.0
    cols = []
    for j in range(2 * T + 1):
        J = O - T + j
        assert r.status[0, 0, j] == 1
        bx0, by0, bx1, by1 = r.box[0, 0, j]
        acc = (r.codes[0, 0, j] & 7) == oracle.CODE_ACCEPT
        # closed form: the plane point seen by pixel q of frame J lies at lateral offset
        # ((J - O) step + (q_x - 32) Z / fx, (q_y - 18) Z / fx) from the axis
        want = []
        for qy in range(c.H):
            for qx in range(c.W):
                dxw = (J - O) * step + (qx - 32) * Z / fx
                dyw = (qy - 18) * Z / fx
                if np.hypot(dxw, dyw) < a:
                    want.append((qx, qy))
        got = [(bx0 + i % 31, by0 + i // 31) for i in np.flatnonzero(acc.reshape(-1))]
        assert sorted(got) == sorted(want), (J, sorted(got), sorted(want))
        cols += [c.clean[J, qy, qx] for qx, qy in want]
    np.testing.assert_allclose(r.rgb[0, 0], np.mean(np.asarray(cols, np.float64), axis=0), atol=1e-12)
    assert r.nacc[0, 0] == len(cols)


def test_pixel_footprint_weight_and_cone_slope_against_thin_lens_render():
    """With exact geometry on a textured plane out of focus, the cone gather approximates the
    thin-lens render (an independent ray-traced simulation of the same lens) far better than the
    pinhole image does, and a cone with the wrong slope does worse."""
    c = synth.make_clip("exact_shift", 65, 37, 31, seed=2)
    fx, Z = c.K[0, 0, 0], float(c.depth[0, 0, 0])
    z0, A, O, T = 0.5 * Z, 0.15, 15, 15
    objs, _, _ = synth.scene_and_path("exact_shift", 65, 37, 31, 2)
    lens = synth.render_thinlens(objs, c.K[O:O + 1], c.w2c_true[O:O + 1], c.W, c.H, A, z0, n_lens=256)[0]
    crop = (20, 10, 25, 17)
    x0, y0, cw, ch = crop
    ref = lens[y0:y0 + ch, x0:x0 + cw]
    psnr = lambda a, b: 10 * np.log10(1.0 / np.mean((np.asarray(a, np.float64) - b) ** 2))
    prm = oracle.Params(mode=oracle.MODE_APERTURE, k=7, T=T, aperture=A, focal_depth=z0, lens_samples=16, cap=31)
    good = oracle.gather_filter(oracle.ClipView.of(c), prm, O, crop=crop).rgb
    wrong = oracle.gather_filter(oracle.ClipView.of(c), oracle.Params(**{**prm.__dict__, "aperture": 2.5 * A}), O,
                                 crop=crop).rgb
    pin = c.clean[O, y0:y0 + ch, x0:x0 + cw]
    assert psnr(good, ref) > psnr(pin, ref) + 3.0
    assert psnr(good, ref) > psnr(wrong, ref) + 3.0


def test_box_scan_equals_brute_force_cone_scan():
    c = synth.make_clip("planes3", 80, 45, 7, seed=4)
    med = oracle.median_depth(c.depth)
    prm = oracle.Params(mode=oracle.MODE_APERTURE, k=7, T=3, aperture=0.05, focal_depth=med, lens_samples=16, cap=31)
    v = oracle.ClipView.of(c)
    O = 3
    r = oracle.gather_filter(v, prm, O, membership=True)
    rng = np.random.default_rng(0)
    full = 0
    for _ in range(40):
        u, w_ = int(rng.integers(0, c.W)), int(rng.integers(0, c.H))
        for j in range(2 * prm.T + 1):
            J = O - prm.T + j
            if r.status[w_, u, j] != 1:
                continue
            brute = oracle.bruteforce(v, prm, O, u, w_, J)
            bx0, by0, bx1, by1 = r.box[w_, u, j]
            acc = (r.codes[w_, u, j] & 7) == oracle.CODE_ACCEPT
            win = np.zeros_like(brute)
            for i in np.flatnonzero(acc.reshape(-1)):
                win[by0 + i // 31, bx0 + i % 31] = 1
            assert (win <= brute).all()
            ys, xs = np.nonzero(brute)
            inside = (xs >= bx0) & (xs <= bx1) & (ys >= by0) & (ys <= by1)
            if inside.all():
                full += 1
                np.testing.assert_array_equal(win, brute)
    assert full > 50


def test_aperture_gauge_and_scale_invariance():
    c = synth.make_clip("planes3", 64, 36, 5, seed=6)
    med = oracle.median_depth(c.depth)
    prm = oracle.Params(mode=oracle.MODE_APERTURE, k=7, T=2, aperture=0.05, focal_depth=med, a0=0.004, cap=21)
    base = oracle.gather_filter(oracle.ClipView.of(c), prm, 2)
    rng = np.random.default_rng(3)
    Rg, tg = synth.rodrigues(rng.normal(0, 0.6, 3)), rng.normal(0, 2.0, 3)
    w2 = np.empty_like(c.w2c)
    for f in range(c.F):
        R, t = c.w2c[f, :, :3], c.w2c[f, :, 3]
        w2[f, :, :3] = R @ Rg.T
        w2[f, :, 3] = t - R @ Rg.T @ tg
    g = oracle.gather_filter(oracle.ClipView(c.rgb, c.depth, c.K, w2), prm, 2)
    np.testing.assert_array_equal(base.nacc, g.nacc)
    np.testing.assert_allclose(base.rgb, g.rgb, atol=1e-9)
    s = 4.0
    w3 = c.w2c.copy()
    w3[:, :, 3] *= s
    p3 = oracle.Params(**{**prm.__dict__, "aperture": prm.aperture * s, "focal_depth": prm.focal_depth * s,
                          "a0": prm.a0 * s})
    sc = oracle.gather_filter(oracle.ClipView(c.rgb, c.depth * s, c.K, w3), p3, 2)
    np.testing.assert_array_equal(base.nacc, sc.nacc)
    np.testing.assert_allclose(base.rgb, sc.rgb, atol=1e-9)
