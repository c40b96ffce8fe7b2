"""Pins of the learned scorer's oracle (CPU only).

The oracle restates the network (three kernel-7 convolutions with ReLU, a 1x1
head) and its weighted cross-entropy with the gradient by the chain rule.  It
is pinned here against things other than itself: finite differences of the
binary64 network, closed forms of hand-set networks (tap direction, zero
padding, channel order), the loss of a constant network, and the bound the
bfloat16 rounding puts between the two modes.
"""
import math

import numpy as np
import pytest

import oracle as orc

W_SMALL, H_SMALL, Y_ROW = 24, 20, 7


def _strip(seed, W=W_SMALL):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, (3, W, 3), dtype=np.uint8)


def _params(seed, scale=0.15):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(orc.SC_NPARAM) * scale).astype(np.float32)
    return p


def test_features_closed_form():
    s = np.zeros((3, 8, 3), np.uint8)
    s[1, 0] = (255, 0, 0)
    s[0, 3] = (10, 20, 30)
    s[2, 7] = (128, 128, 128)
    f = orc.sc_features(s, y=5, H=11, mixed=False)
    luma_red = (77 * 255 + 128) >> 8
    assert f[0, 4] == (luma_red - 128) / 128 and f[0, 5] == (255 - 128) / 128
    assert f[0, 6] == -1.0 and f[0, 7] == -1.0
    assert f[3, 1] == (10 - 128) / 128 and f[3, 2] == (20 - 128) / 128 and f[3, 3] == (30 - 128) / 128
    assert f[7, 8] == 0.0 and f[7, 9] == 0.0
    assert f[0, 12] == (0 - 3.5) / 8 and f[7, 12] == (7 - 3.5) / 8
    assert np.all(f[:, 13] == (5 - 5.0) / 11)
    fm = orc.sc_features(s, y=5, H=11, mixed=True)
    assert np.array_equal(fm[:, :12], f[:, :12])          # (v - 128) / 128 is exact in bf16
    assert np.all(np.abs(fm[:, 12:] - f[:, 12:]) <= 2.0 ** -9)


@pytest.mark.parametrize("mode", [orc.SC_EXACT, orc.SC_MIXED])
def test_hand_set_network_shift_and_padding(mode):
    """Layer 1 takes the middle-row luma at x+1 (tap 4), layers 2-3 pass
    channel 0 through (tap 3), the head reads channel 0: the logit is
    relu((Y[x+1] - 128) / 128), and 0 at the last column (zero padding)."""
    off = orc.sc_offsets()
    p = np.zeros(orc.SC_NPARAM, np.float32)
    p[off["W1"] + (0 * 14 + 4) * 7 + 4] = 1.0
    p[off["W2"] + (0 * 32 + 0) * 7 + 3] = 1.0
    p[off["W3"] + (0 * 32 + 0) * 7 + 3] = 1.0
    p[off["wh"] + 0] = 1.0
    s = _strip(3, 16)
    lg = orc.sc_forward(s, 5, 12, p, mode=mode)
    Y = np.array([orc.luma(*s[1, x]) for x in range(16)])
    want = np.maximum((Y[1:] - 128) / 128.0, 0.0)
    assert np.array_equal(lg[:-1], want) and lg[-1] == 0.0
    # the same through tap 2 reads x-1, and column 0 sees the zero padding
    p2 = p.copy()
    p2[off["W1"] + (0 * 14 + 4) * 7 + 4] = 0.0
    p2[off["W1"] + (0 * 14 + 4) * 7 + 2] = 1.0
    lg2 = orc.sc_forward(s, 5, 12, p2, mode=mode)
    assert lg2[0] == 0.0 and np.array_equal(lg2[1:], np.maximum((Y[:-1] - 128) / 128.0, 0.0))


def test_constant_network_loss_closed_form():
    off = orc.sc_offsets()
    p = np.zeros(orc.SC_NPARAM, np.float32)
    b = 0.75
    p[off["bh"]] = b
    lab = np.zeros(W_SMALL, np.uint8)
    lab[[3, 4, 17]] = 1
    pw = 5.0
    loss, g = orc.sc_loss_grad(_strip(1), Y_ROW, H_SMALL, lab, p, pos_weight=pw,
                               mode=orc.SC_EXACT)
    sp = math.log1p(math.exp(b))
    w = np.where(lab == 1, pw, 1.0)
    assert loss == pytest.approx(float((w * (sp - lab * b)).sum()), rel=1e-12)
    sig = 1.0 / (1.0 + math.exp(-b))
    assert g[off["bh"]] == pytest.approx(float((w * (sig - lab)).sum()), rel=1e-12)
    assert np.all(g[:off["bh"]] == 0.0)   # every activation is 0: no other gradient


def test_gradient_matches_finite_differences():
    """Every parameter block, central differences of the binary64 network."""
    s = _strip(11)
    p = _params(12)
    lab = (np.random.default_rng(13).uniform(size=W_SMALL) < 0.25).astype(np.uint8)
    _, g = orc.sc_loss_grad(s, Y_ROW, H_SMALL, lab, p, pos_weight=3.0, mode=orc.SC_EXACT)
    off = orc.sc_offsets()
    rng = np.random.default_rng(14)
    bounds = list(off.values()) + [orc.SC_NPARAM]
    idx = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        idx += list(rng.integers(a, b, size=min(6, b - a)))
    for i in idx:
        h = 1e-6 * max(1.0, abs(float(p[i])))   # small: no ReLU kink crossed
        # the parameters are binary32: step to the neighbouring representable
        # values and divide by the true step
        hp = np.float32(p[i] + h) - p[i]
        hm = p[i] - np.float32(p[i] - h)
        q = p.copy(); q[i] = p[i] + hp
        lp, _ = orc.sc_loss_grad(s, Y_ROW, H_SMALL, lab, q, 3.0, orc.SC_EXACT)
        q[i] = p[i] - hm
        lm, _ = orc.sc_loss_grad(s, Y_ROW, H_SMALL, lab, q, 3.0, orc.SC_EXACT)
        fd = (lp - lm) / (float(hp) + float(hm))
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_mixed_mode_stays_near_exact():
    """bfloat16 features, weights and activations move the logits by a few
    bf16 steps at most, and the gradient direction is kept."""
    s = _strip(21, 64)
    p = _params(22, 0.1)
    le = orc.sc_forward(s, 30, 100, p, mode=orc.SC_EXACT)
    lm = orc.sc_forward(s, 30, 100, p, mode=orc.SC_MIXED)
    assert np.max(np.abs(le - lm)) < 0.05
    lab = np.zeros(64, np.uint8)
    lab[[10, 40]] = 1
    _, ge = orc.sc_loss_grad(s, 30, 100, lab, p, 4.0, orc.SC_EXACT)
    _, gm = orc.sc_loss_grad(s, 30, 100, lab, p, 4.0, orc.SC_MIXED)
    cos = float(ge @ gm / (np.linalg.norm(ge) * np.linalg.norm(gm)))
    assert cos > 0.999
    assert np.max(np.abs(ge - gm)) < 0.03 * np.max(np.abs(ge))


def test_bf16_rounding_is_round_to_nearest_even():
    assert orc.bf16(1.0) == 1.0
    assert orc.bf16(1.0 + 2.0 ** -8) == 1.0                       # tie -> even
    assert orc.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie -> even (up)
    assert orc.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert orc.bf16(-2.5) == -2.5


def test_fit_from_candidates_equals_estimate():
    """orc_fit on the candidate list of orc_candidates gives orc_estimate's result."""
    from paper_2210_14771_gb300 import synth
    f, _ = synth.frame(5, 1, 240, 320, "centred")
    p = orc.params(n_strips=16, cands_per_strip=4, n_hyps=128, seed=3)
    xs, ys, ss = orc.candidates(f, p)
    r1, _ = orc.estimate(f, 99, p)
    r2 = orc.fit(xs, ys, ss, 240, 320, 99, p)
    assert r1 == r2


def _by_half(xs, ys, rows, W):
    """Candidate points grouped by (strip, half): {(i, half): [(x, y), ...]}."""
    out = {}
    for x, y in zip(xs.tolist(), ys.tolist()):
        i = int(np.nonzero(rows == y)[0][0])
        out.setdefault((i, int(x >= W // 2)), []).append((x, y))
    return out


@pytest.mark.parametrize("K", [2, 4])
def test_learned_fallback_rule_boundary(K):
    """The fallback rule of the learned candidates (Sec. 2.2.4's scorer with
    the handcrafted extractor as fallback below p = 1/2): a half-strip whose
    best learned Q15 score is 16383 takes the handcrafted points of that half,
    one whose best is 16384 keeps its learned point, and no other half
    changes.  Expectations are written from the rule itself: the learned
    point is the hand-placed peak of that half; the handcrafted points are the
    oracle's own handcrafted candidates of that half."""
    from paper_2210_14771_gb300 import synth
    H, W = 480, 640
    frame, _ = synth.frame(0, 0, H, W)
    p = orc.params(n_strips=16, cands_per_strip=K)
    rows = orc.strip_rows(H, 16, p.alpha)
    hand = _by_half(*orc.candidates(frame, p)[:2], rows, W)
    learned = np.zeros((16, W), np.uint16)
    peaks = {}
    rng = np.random.default_rng(5)
    for i in range(16):
        for half in (0, 1):
            lo, hi = (10, W // 2 - 10) if half == 0 else (W // 2 + 10, W - 10)
            x = int(rng.integers(lo, hi))
            # alternate the two boundary values and a clearly confident peak
            v = (16383, 16384, 30000)[(2 * i + half) % 3]
            learned[i, x] = v
            peaks[(i, half)] = (x, int(rows[i]), v)
    for fallback in (False, True):
        xs, ys, ss = orc.learned_candidates(frame, learned, fallback, p)
        got = _by_half(xs, ys, rows, W)
        for (i, half), (x, y, v) in peaks.items():
            if fallback and v < 16384:
                want = hand.get((i, half), [])
            else:
                want = [(x, y)]   # later picks (K = 4) score 0 and are dropped by t_ps
            assert got.get((i, half), []) == want, (fallback, i, half, v)
        # the scores carried along are the learned ones where the learned point is kept
        kept = {(x, y): s for x, y, s in zip(xs.tolist(), ys.tolist(), ss.tolist())}
        for (i, half), (x, y, v) in peaks.items():
            if not (fallback and v < 16384):
                assert kept[(x, y)] == v


def test_learned_fallback_all_unsure_is_handcrafted():
    """With every learned score below one half the fallback gives exactly the
    handcrafted candidates, in order; without it nothing survives t_ps."""
    from paper_2210_14771_gb300 import synth
    H, W = 480, 640
    frame, _ = synth.frame(1, 3, H, W)
    p = orc.params(n_strips=16, cands_per_strip=2)
    learned = np.full((16, W), 500, np.uint16)   # p ~ 0.015 everywhere: below t_ps too
    hx, hy, hs = orc.candidates(frame, p)
    fx, fy, fs = orc.learned_candidates(frame, learned, True, p)
    assert np.array_equal(hx, fx) and np.array_equal(hy, fy) and np.array_equal(hs, fs)
    nx, _, _ = orc.learned_candidates(frame, learned, False, p)
    assert len(nx) == 0
