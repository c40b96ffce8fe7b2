"""Pins of the oracle of the paper's own learned scorer (Sec. 2.2.4: 3x3
convolutions to 8, 16, 32 features, ReLU, 1x1 head, sigmoid, on RGBXY strips
7 rows high): gradient against finite differences, the 7 x 7 receptive
field, a hand-set network with a closed-form output, mirror symmetry, the
constant network's loss and the soft targets."""
import math

import numpy as np
import pytest

import oracle as orc

H, W = 40, 48


def _params(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(orc.SC2_NPARAM) * scale).astype(np.float32)


def _strip(seed, y=20):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    return f, orc.sc2_strip(f, y)


def test_layout_and_strip_rows():
    o = orc.sc2_offsets()
    assert (o["b1"], o["W2"], o["b2"], o["W3"], o["b3"], o["wh"], o["bh"]) == \
        (360, 368, 1520, 1536, 6144, 6176, 6208)
    f, (rgb7, rows) = _strip(1, y=1)
    assert rows.tolist() == [0, 0, 0, 1, 2, 3, 4]            # clamped at the top
    assert np.array_equal(rgb7[3], f[1]) and np.array_equal(rgb7[0], f[0])
    _, (_, rows) = _strip(1, y=H - 2)
    assert rows.tolist() == [H - 5, H - 4, H - 3, H - 2, H - 1, H - 1, H - 1]


@pytest.mark.parametrize("pw", [1.0, 6.0])
def test_gradient_matches_finite_differences(pw):
    _, (rgb7, rows) = _strip(2)
    p = _params(3)
    t = np.random.default_rng(4).random(W)
    _, g = orc.sc2_loss_grad(rgb7, rows, H, t, p, pw)
    o = orc.sc2_offsets()
    rng = np.random.default_rng(5)
    blocks = [(o["W1"], o["b1"]), (o["b1"], o["W2"]), (o["W2"], o["b2"]), (o["b2"], o["W3"]),
              (o["W3"], o["b3"]), (o["b3"], o["wh"]), (o["wh"], o["bh"]), (o["bh"], o["bh"] + 1)]
    h = 2.0 ** -16
    for a, b in blocks:
        for i in rng.choice(np.arange(a, b), size=min(6, b - a), replace=False):
            pp, pm = p.copy(), p.copy()
            pp[i] = np.float32(p[i] + h)
            pm[i] = np.float32(p[i] - h)
            lp, _ = orc.sc2_loss_grad(rgb7, rows, H, t, pp, pw)
            lm, _ = orc.sc2_loss_grad(rgb7, rows, H, t, pm, pw)
            fd = (lp - lm) / (float(pp[i]) - float(pm[i]))
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (a, i, fd, g[i])


def test_receptive_field_is_7_by_7():
    f, (rgb7, rows) = _strip(6)
    p = _params(7)
    base = orc.sc2_forward(rgb7, rows, H, p)
    x = 20
    for dx, inside in ((4, False), (-4, False), (3, True), (-3, True)):
        for k in (0, 6):
            m = rgb7.copy()
            m[k, x + dx] = 255 - m[k, x + dx]
            out = orc.sc2_forward(m, rows, H, p)
            assert (out[x] != base[x]) == inside, (dx, k)


def test_hand_set_network_passes_the_red_channel_of_the_middle_pixel():
    f, (rgb7, rows) = _strip(8)
    p = np.zeros(orc.SC2_NPARAM, np.float32)
    o = orc.sc2_offsets()
    p[o["W1"] + ((0 * 5 + 0) * 3 + 1) * 3 + 1] = 1.0     # W1[0][R][1][1]
    p[o["W2"] + ((0 * 8 + 0) * 3 + 1) * 3 + 1] = 1.0     # W2[0][0][1][1]
    p[o["W3"] + ((0 * 16 + 0) * 3 + 1) * 3 + 1] = 1.0    # W3[0][0][1][1]
    p[o["wh"]] = 1.0
    out = orc.sc2_forward(rgb7, rows, H, p)
    want = np.maximum(0.0, (f[20, :, 0].astype(np.float64) - 128) / 128)
    assert np.array_equal(out, want)


def test_mirror_symmetry():
    """Mirrored strip, mirrored kernels and a negated X weight: mirrored logits."""
    f, (rgb7, rows) = _strip(9)
    p = _params(10)
    o = orc.sc2_offsets()
    q = p.copy()
    for (wk, cout, cin) in (("W1", 8, 5), ("W2", 16, 8), ("W3", 32, 16)):
        w = p[o[wk]:o[wk] + cout * cin * 9].reshape(cout, cin, 3, 3)[..., ::-1].copy()
        if wk == "W1":
            w[:, 3] = -w[:, 3]                                 # X = -X under the mirror
        q[o[wk]:o[wk] + cout * cin * 9] = w.reshape(-1)
    a = orc.sc2_forward(rgb7, rows, H, p)
    b = orc.sc2_forward(np.ascontiguousarray(rgb7[:, ::-1]), rows, H, q)
    assert np.allclose(b[::-1], a, rtol=0, atol=1e-12)


def test_constant_network_loss_and_bias_gradient():
    _, (rgb7, rows) = _strip(11)
    t = np.random.default_rng(12).random(W)
    loss, g = orc.sc2_loss_grad(rgb7, rows, H, t, np.zeros(orc.SC2_NPARAM, np.float32))
    assert loss == pytest.approx(W * math.log(2.0), rel=1e-15)
    assert g[orc.sc2_offsets()["bh"]] == pytest.approx(float((0.5 - t).sum()), abs=1e-12)
    assert not np.any(g[:orc.sc2_offsets()["bh"]])      # dead ReLUs: nothing else moves


def test_weighted_constant_network_closed_form():
    """Column x counts 1 + (pw - 1) t_x times: for the zero network (p = 1/2
    everywhere) the loss is log 2 sum_x w_x and the head-bias gradient
    sum_x w_x (1/2 - t_x)."""
    _, (rgb7, rows) = _strip(13)
    t = np.random.default_rng(14).random(W)
    pw = 9.0
    w = 1.0 + (pw - 1.0) * t
    loss, g = orc.sc2_loss_grad(rgb7, rows, H, t, np.zeros(orc.SC2_NPARAM, np.float32), pw)
    assert loss == pytest.approx(math.log(2.0) * float(w.sum()), rel=1e-14)
    assert g[orc.sc2_offsets()["bh"]] == pytest.approx(float((w * (0.5 - t)).sum()), abs=1e-11)


def test_soft_targets():
    y = 10
    t = orc.sc2_targets(30.0, 10.0, 5.0, 1, 64, y, 3.0)   # circle crosses row 10 at x = 25, 35
    assert t[25] == 1.0 and t[35] == 1.0
    assert t[28] == pytest.approx(math.exp(-0.5), rel=1e-12)   # 3 px inside: d = sigma
    assert np.all(t >= 0) and np.all(t <= 1)
    assert not np.any(orc.sc2_targets(30.0, 10.0, 5.0, 0, 64, y, 3.0))


def test_mixed_mode_is_exact_when_nothing_rounds():
    """The hand-set identity network moves bfloat16-exact colours (k / 128)
    through bfloat16-exact unit weights: the mixed mode equals the exact one."""
    f, (rgb7, rows) = _strip(13)
    p = np.zeros(orc.SC2_NPARAM, np.float32)
    o = orc.sc2_offsets()
    p[o["W1"] + ((0 * 5 + 1) * 3 + 1) * 3 + 1] = 1.0     # green channel this time
    p[o["W2"] + ((0 * 8 + 0) * 3 + 1) * 3 + 1] = 1.0
    p[o["W3"] + ((0 * 16 + 0) * 3 + 1) * 3 + 1] = 1.0
    p[o["wh"]] = 1.0
    a = orc.sc2_forward(rgb7, rows, H, p)
    b = orc.sc2_forward(rgb7, rows, H, p, mixed=True)
    assert np.array_equal(a, b)
    assert np.array_equal(a, np.maximum(0.0, (f[20, :, 1].astype(np.float64) - 128) / 128))


def test_mixed_mode_within_the_bfloat16_bound():
    """Random networks: bfloat16 weights, features and activations move a
    logit by a few 2^-8 relative steps of the magnitudes it sums; the mode
    stays within 0.05 (1 + |logit|) of the exact network and is not equal to it."""
    _, (rgb7, rows) = _strip(14)
    for seed in range(3):
        p = _params(15 + seed, scale=0.2)
        a = orc.sc2_forward(rgb7, rows, H, p)
        b = orc.sc2_forward(rgb7, rows, H, p, mixed=True)
        assert np.all(np.abs(a - b) <= 0.05 * (1.0 + np.abs(a)))
        assert not np.array_equal(a, b)
