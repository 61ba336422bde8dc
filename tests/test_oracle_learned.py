"""Pins of the oracle's learned per-sample weighting (samples, features, MLP, loss gradients)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def tiny():
    c = synth.make_clip("planes3", 64, 36, 9, seed=7)
    v = oracle.ClipView.of(c)
    prm = oracle.default_params(c.depth, k=5, T=4)
    return c, v, prm


def test_zero_head_gives_the_mean_of_the_capped_set(tiny):
    c, v, prm = tiny
    feat, col, n, plain = oracle.learned_crop(v, prm, 4, crop=(10, 8, 6, 5))
    W1, b1, W2, b2 = oracle.he_init(1)
    for y in range(5):
        for x in range(6):
            ol, of, conf, _ = oracle.mlp_pixel(feat[y, x], col[y, x], n[y, x], W1, b1, 0 * W2, 0 * b2, plain=plain[y, x])
            np.testing.assert_allclose(ol, col[y, x, :n[y, x]].mean(0), atol=1e-12)
            assert conf == pytest.approx(0.5)
            np.testing.assert_allclose(of, ol)  # conf >= 0.5 keeps the learned result


def test_low_confidence_falls_back_to_the_plain_filter(tiny):
    c, v, prm = tiny
    crop = (0, 0, 64, 36)
    feat, col, n, plain = oracle.learned_crop(v, prm, 4, crop=crop)
    np.testing.assert_allclose(plain, oracle.gather_filter(v, prm, 4, crop=crop).rgb, atol=1e-15)
    W1, b1, W2, b2 = oracle.he_init(2)
    b2 = np.array([0.0, -30.0])
    W2 = W2.copy()
    W2[1] = 0.0
    for y, x in [(0, 0), (17, 31), (35, 63)]:
        _, of, conf, _ = oracle.mlp_pixel(feat[y, x], col[y, x], n[y, x], W1, b1, W2, b2, plain=plain[y, x])
        assert conf < 1e-9
        np.testing.assert_array_equal(of, plain[y, x])


def test_features_in_canonical_order_have_the_closed_form_on_exact_shift():
    """One sample per frame, at distance 0, depth residual 0, same colour as the reference; frames
    in the order O, O-1, O+1, ...; the Eq. 4 log weight reduces to the frame term."""
    c = synth.make_clip("exact_shift", 64, 36, 11, seed=3)
    v = oracle.ClipView.of(c)
    O, T = 5, 5
    prm = oracle.default_params(c.depth, k=5, T=T)
    feat, col, n, plain = oracle.learned_crop(v, prm, O, crop=(30, 10, 1, 1))
    f, cc, nn = feat[0, 0], col[0, 0], n[0, 0]
    order = [0, -1, 1, -2, 2, -3, 3, -4, 4, -5, 5]
    assert nn == len(order)
    for s, dJ in enumerate(order):
        want_col = c.clean[O + dJ, 10, 30 - dJ]
        np.testing.assert_allclose(cc[s], want_col, atol=0)
        np.testing.assert_allclose(f[s, :3], want_col, atol=0)
        np.testing.assert_allclose(f[s, 3:6], 0.0, atol=1e-12)
        assert f[s, 6] == pytest.approx(0.0, abs=1e-9)
        assert f[s, 7] == pytest.approx(dJ / T)
        assert f[s, 8] == pytest.approx(0.0, abs=1e-9)
        assert f[s, 9] == pytest.approx(-dJ ** 2 / (2 * prm.sigma_f ** 2), abs=1e-12)
        assert f[s, 10] == 1.0 and f[s, 11] == nn / 64.0 and f[s, 15] == 0.0
        # every sample has the reference's colour, so the plain result does too
        np.testing.assert_allclose(f[s, 12:15], 0.0, atol=1e-12)


def test_set_size_feature_is_the_whole_gathered_set(tiny):
    c, v, prm = tiny
    feat, col, n, plain = oracle.learned_crop(v, prm, 4, crop=(0, 0, 64, 36))
    full = oracle.gather_filter(v, prm, 4)
    has = n > 0
    np.testing.assert_array_equal(feat[..., 0, 11][has], full.nacc[has] / 64.0)


def test_plain_residual_features_against_the_filter_output(tiny):
    """Features 12-14 are each sample's colour minus the plain Eq. 4 output of the whole set:
    checked against the gather-and-filter's own output and the stored sample colours."""
    c, v, prm = tiny
    feat, col, n, plain = oracle.learned_crop(v, prm, 4, crop=(0, 0, 64, 36))
    full = oracle.gather_filter(v, prm, 4)
    m = np.arange(64)[None, None, :] < n[..., None]
    resid = col - full.rgb[:36, :64][:, :, None, :]
    np.testing.assert_allclose(feat[..., 12:15][m], resid[m], atol=1e-12, rtol=0)
    assert (feat[..., 15] == 0).all()
    assert np.abs(feat[..., 12:15][m]).max() > 0.01


def test_cap_keeps_the_first_64_in_canonical_order():
    c = synth.make_clip("exact_const", 48, 27, 9, seed=0)
    v = oracle.ClipView.of(c)
    prm = oracle.default_params(c.depth, k=7, T=4, radius_rel=0.05)  # wide gate: many samples
    feat, col, n, plain = oracle.learned_crop(v, prm, 4, crop=(20, 12, 4, 3))
    full = oracle.gather_filter(v, prm, 4, crop=(20, 12, 4, 3))
    assert (full.nacc > 64).all()
    assert (n == 64).all()
    np.testing.assert_array_equal(feat[:, :, :, 11], np.repeat((full.nacc / 64.0)[..., None], 64, -1))
    rank = {0: 0, -1: 1, 1: 2, -2: 3, 2: 4, -3: 5, 3: 6, -4: 7, 4: 8}
    for y in range(3):
        for x in range(4):
            r = [rank[int(round(t * 4))] for t in feat[y, x, :, 7]]
            assert r == sorted(r)


def test_softplus_weights_and_sigmoid_confidence_against_scipy():
    from scipy.special import expit
    # two samples whose only non-zero feature is the red channel; h0 = ReLU(2 f0), z = (3 h0 - 1, -h0)
    feat = np.zeros((2, 16))
    feat[:, 0] = [0.25, 0.75]
    col = np.array([[0.25, 0.1, 0.2], [0.75, 0.4, 0.9]])
    W1 = np.zeros((64, 16)); W1[0, 0] = 2.0
    W2 = np.zeros((2, 64)); W2[0, 0] = 3.0; W2[1, 0] = -1.0
    b1, b2 = np.zeros(64), np.array([-1.0, 0.0])
    ol, of, conf, z = oracle.mlp_pixel(feat, col, 2, W1, b1, W2, b2, round_bf16=False)
    zw = 3 * 2 * feat[:, 0] - 1
    w = np.logaddexp(0.0, zw)
    np.testing.assert_allclose(z[:, 0], zw, atol=1e-15)
    np.testing.assert_allclose(ol, (w[:, None] * col).sum(0) / w.sum(), atol=1e-14)
    assert conf == pytest.approx(expit(-2 * feat[:, 0]).mean(), abs=1e-15)


def test_bf16_mode_rounds_inputs_weights_and_hidden_activations():
    """round_bf16: features, W1, W2 and the ReLU output enter the products as BF16 (8 significant
    bits, round to nearest even); b1, b2 as FP32.  One sample, one hidden unit, closed forms."""
    feat = np.zeros((1, 16))
    col = np.array([[0.5, 0.5, 0.5]])
    W1 = np.zeros((64, 16))
    W2 = np.zeros((2, 64)); W2[0, 0] = 1.0
    b1, b2 = np.zeros(64), np.zeros(2)
    # h = 1 + 2^-10 is not a BF16 value: it rounds to 1 (z_w exactly 1), or is kept (z_w = h)
    feat[0, 10] = 1.0
    b1[0] = 1.0 + 2.0 ** -10
    z_r = oracle.mlp_pixel(feat, col, 1, W1, b1, W2, b2, round_bf16=True)[3]
    z_f = oracle.mlp_pixel(feat, col, 1, W1, b1, W2, b2, round_bf16=False)[3]
    assert z_r[0, 0] == 1.0 and z_f[0, 0] == 1.0 + 2.0 ** -10
    # a tie between two BF16 values rounds to the even one: 1 + 3 * 2^-8 -> 1 + 2^-6
    b1[0] = 1.0 + 3 * 2.0 ** -8
    assert oracle.mlp_pixel(feat, col, 1, W1, b1, W2, b2, round_bf16=True)[3][0, 0] == 1.0 + 2.0 ** -6
    # a feature and a weight are rounded too: f = 1 + 2^-9 (down to 1), W1 = 3 + 3 * 2^-8 (up to 3 + 2^-6)
    b1[0] = 0.0
    feat[0, 10] = 0.0
    feat[0, 3] = 1.0 + 2.0 ** -9
    W1[0, 3] = 3.0 + 3 * 2.0 ** -8
    z = oracle.mlp_pixel(feat, col, 1, W1, b1, W2, b2, round_bf16=True)[3][0, 0]
    assert z == 3.0 + 2.0 ** -6
    # W2 likewise: 1 + 2^-9 rounds to 1
    W2[0, 0] = 1.0 + 2.0 ** -9
    assert oracle.mlp_pixel(feat, col, 1, W1, b1, W2, b2, round_bf16=True)[3][0, 0] == 3.0 + 2.0 ** -6


def test_gradients_match_central_differences(tiny):
    c, v, _ = tiny
    prm = oracle.default_params(c.depth, k=5, T=4, radius_rel=0.03)  # a wider gate: several samples per pixel
    feat, col, n, plain = oracle.learned_crop(v, prm, 4, crop=(20, 10, 8, 6))
    P = 48
    feat, col, n, plain = feat.reshape(P, 64, 16), col.reshape(P, 64, 3), n.reshape(P), plain.reshape(P, 3)
    clean = c.clean[4, 10:16, 20:28].reshape(P, 3).astype(np.float64)
    # pixels with a single sample have learned == plain, so their BCE target sits on its step
    keep = n >= 3
    feat, col, n, plain, clean = feat[keep], col[keep], n[keep], plain[keep], clean[keep]
    assert len(n) >= 10
    W1, b1, W2, b2 = oracle.he_init(5)
    b2 = np.array([0.3, 0.1])
    L, gW1, gb1, gW2, gb2 = oracle.mlp_loss_grad(feat, col, n, plain, clean, W1, b1, W2, b2, round_bf16=False)
    params = [W1, b1, W2, b2]
    grads = [gW1, gb1, gW2, gb2]
    rng = np.random.default_rng(0)
    eps = 1e-6
    checked = 0
    for pi, (P_, G_) in enumerate(zip(params, grads)):
        idx = [tuple(int(rng.integers(0, s)) for s in P_.shape) for _ in range(12)]
        for ix in idx:
            Pp, Pm = [q.copy() for q in params], [q.copy() for q in params]
            Pp[pi][ix] += eps
            Pm[pi][ix] -= eps
            Lp = oracle.mlp_loss_grad(feat, col, n, plain, clean, *Pp, round_bf16=False)[0]
            Lm = oracle.mlp_loss_grad(feat, col, n, plain, clean, *Pm, round_bf16=False)[0]
            fwd, bwd = (Lp - L) / eps, (L - Lm) / eps
            if abs(fwd - bwd) > 1e-3 * max(1.0, abs(fwd)):
                continue  # a ReLU kink or a flip of the (constant) BCE target inside the step
            fd = (Lp - Lm) / (2 * eps)
            assert G_[ix] == pytest.approx(fd, rel=1e-4, abs=1e-9), (pi, ix)
            checked += 1
    assert checked >= 40


def test_gradient_term_scales_bound_the_gradients(tiny):
    """The per-entry sums of |term| that the GPU gradient tolerance is scaled by: they bound the
    gradients (triangle inequality), and for one pixel with one sample and a positive hidden unit
    each entry has a single term, so the two are equal in magnitude (layer 2 and b1 of that
    unit); doubling the batch by repeating its pixels leaves them unchanged (both are means)."""
    c, v, _ = tiny
    prm = oracle.default_params(c.depth, k=5, T=4, radius_rel=0.03)
    feat, col, n, plain = oracle.learned_crop(v, prm, 4, crop=(20, 10, 8, 6))
    P = 48
    feat, col, n, plain = feat.reshape(P, 64, 16), col.reshape(P, 64, 3), n.reshape(P), plain.reshape(P, 3)
    clean = c.clean[4, 10:16, 20:28].reshape(P, 3).astype(np.float64)
    W1, b1, W2, b2 = oracle.he_init(5)
    b2 = np.array([0.3, 0.1])
    out = oracle.mlp_loss_grad(feat, col, n, plain, clean, W1, b1, W2, b2, term_scale=True)
    for g, a in zip(out[1:5], out[5:9]):
        assert (np.abs(g) <= a * (1 + 1e-12) + 1e-300).all()
        assert (a >= 0).all()
    assert out[5].max() > 0 and out[7].max() > 0
    out2 = oracle.mlp_loss_grad(np.concatenate([feat, feat]), np.concatenate([col, col]), np.concatenate([n, n]),
                                np.concatenate([plain, plain]), np.concatenate([clean, clean]), W1, b1, W2, b2,
                                term_scale=True)
    for x, y in zip(out[1:], out2[1:]):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-300)
    # one pixel, one sample: every entry of gW2, gb2 and gb1 is a single term
    one = [np.where(n >= 1)[0][0]]
    n1 = np.ones(1, np.int32)
    o1 = oracle.mlp_loss_grad(feat[one], col[one], n1, plain[one], clean[one], W1, b1, W2, b2, term_scale=True)
    for g, a in ((o1[2], o1[6]), (o1[3], o1[7]), (o1[4], o1[8])):
        np.testing.assert_allclose(np.abs(g), a, rtol=1e-12, atol=1e-300)


def test_depth_residual_feature_sign_and_size():
    """Raising the depth of every other frame by delta < r keeps each sample (it moves along its
    own ray, still inside the gate) and makes its depth residual exactly +delta."""
    c = synth.make_clip("exact_shift", 64, 36, 7, seed=3)
    O, T = 3, 3
    prm = oracle.default_params(c.depth, k=5, T=T)
    delta = np.float32(0.25 * prm.radius)
    depth = c.depth.copy()
    for J in range(c.F):
        if J != O:
            depth[J] += delta
    v = oracle.ClipView(c.rgb, depth, c.K, c.w2c)
    feat, col, n, plain = oracle.learned_crop(v, prm, O, crop=(30, 10, 1, 1))
    f = feat[0, 0]
    assert n[0, 0] == 2 * T + 1
    assert f[0, 8] == pytest.approx(0.0, abs=1e-9)
    d_exact = float(np.float32(c.depth[1, 0, 0] + delta)) - float(c.depth[1, 0, 0])
    for s in range(1, 2 * T + 1):
        assert f[s, 8] == pytest.approx(d_exact / prm.radius, rel=1e-6)
        assert f[s, 6] >= abs(f[s, 8]) - 1e-12
