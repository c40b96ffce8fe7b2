"""Pins of the oracle's temporal smoothing of a stream's results (CPU):
memoryless at gamma 0, fixed points, scene changes, the hold of a circle
through failed frames, the weighted mean itself and the noise it removes."""
import math
from fractions import Fraction

import numpy as np

import oracle as orc


def _r(cx, cy, r, score=0.5, valid=1, n=10):
    return (cx, cy, r, score, valid, n)


def test_gamma_zero_is_memoryless():
    rng = np.random.default_rng(1)
    seq = [_r(*rng.uniform(50, 300, 3), rng.uniform(0.05, 1), int(rng.random() < 0.8), 7)
           for _ in range(40)]
    out, _ = orc.smooth_chain(seq, 640, 0.0, 0.05, 0.06)
    for a, b in zip(seq, out):
        if a[4]:
            assert (b["cx"], b["cy"], b["r"], b["valid"]) == \
                (np.float32(a[0]), np.float32(a[1]), np.float32(a[2]), 1)
        else:
            assert b["valid"] == 0


def test_constant_circle_is_a_fixed_point_and_confidence_is_geometric():
    g, s = 0.75, 0.4
    out, st = orc.smooth_chain([_r(200.5, 100.25, 80.0, s)] * 60, 640, g, 0.05, 0.06)
    for o in out:
        assert abs(o["cx"] - 200.5) <= 2e-4 and abs(o["cy"] - 100.25) <= 2e-4
        assert abs(o["r"] - 80.0) <= 2e-4
    # conf_k = s (1 + g + ... + g^k) -> s / (1 - g)
    assert abs(st[3] - s / (1 - g)) < 1e-5


def test_scene_change_resets_to_the_new_circle():
    W = 640
    seq = [_r(200.0, 100.0, 80.0)] * 5 + [_r(200.0 + 0.05 * W + 1.0, 100.0, 80.0, 0.3)]
    out, st = orc.smooth_chain(seq, W, 0.9, 0.05, 0.06)
    assert (out[-1]["cx"], out[-1]["cy"], out[-1]["r"]) == (np.float32(233.0), 100.0, 80.0)
    assert st[3] == np.float32(0.3)
    # just inside the jump distance: a weighted mean, strictly between the two
    seq[-1] = _r(200.0 + 0.05 * W - 1.0, 100.0, 80.0, 0.3)
    out, _ = orc.smooth_chain(seq, W, 0.9, 0.05, 0.06)
    assert 200.0 < out[-1]["cx"] < 231.0


def test_weighted_mean_within_binary32_rounding():
    """Second frame: (d c' + s c) / (d + s) with d = conf gamma, the exact
    rational value within the rounding of four binary32 operations."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = [float(np.float32(v)) for v in rng.uniform(10, 500, 3)]
        b = [float(np.float32(v + rng.uniform(-5, 5))) for v in a]
        s0, s1 = (float(np.float32(v)) for v in rng.uniform(0.05, 1.0, 2))
        g = float(np.float32(rng.uniform(0.1, 0.95)))
        out, _ = orc.smooth_chain([_r(*a, s0), _r(*b, s1)], 4096, g, 0.05, 0.06)
        d = Fraction(float(np.float32(s0 * g)))
        for k, key in enumerate(("cx", "cy", "r")):
            exact = (d * Fraction(a[k]) + Fraction(s1) * Fraction(b[k])) / (d + Fraction(s1))
            assert abs(Fraction(out[1][key]) - exact) <= exact * Fraction(4, 2 ** 23)


def test_hold_through_failed_frames_then_give_up():
    s, g, t_hold = 0.5, 0.8, 0.06
    seq = [_r(150.0, 120.0, 90.0, s)] + [_r(0, 0, 0, 0, 0, 0)] * 15
    out, st = orc.smooth_chain(seq, 640, g, 0.05, t_hold)
    held = [o for o in out[1:] if o["valid"]]
    # held while s g^k >= t_hold: k <= log(t_hold / s) / log(g) = 9.5
    assert len(held) == math.floor(math.log(t_hold / s) / math.log(g))
    assert all((o["cx"], o["cy"], o["r"], o["n_inliers"]) == (150.0, 120.0, 90.0, 0) for o in held)
    assert out[-1]["valid"] == 0 and np.all(st == 0)


def test_smoothing_removes_estimation_noise():
    """Noisy estimates of a static circle (sigma 2 px): the smoothed centre
    errs by about sigma sqrt((1 - g) / (1 + g)) in the steady state."""
    rng = np.random.default_rng(3)
    n, sig, g = 2000, 2.0, 0.8
    seq = [_r(320 + rng.normal(0, sig), 240 + rng.normal(0, sig), 200 + rng.normal(0, sig), 0.5)
           for _ in range(n)]
    out, _ = orc.smooth_chain(seq, 640, g, 0.05, 0.06)
    raw = np.array([[q[0] - 320, q[1] - 240] for q in seq[100:]])
    sm = np.array([[o["cx"] - 320, o["cy"] - 240] for o in out[100:]])
    ratio = np.sqrt((sm ** 2).mean() / (raw ** 2).mean())
    assert abs(ratio - math.sqrt((1 - g) / (1 + g))) < 0.05
