"""Pins of the tracked fit in the oracle (CPU): the previous circle as one
more RANSAC hypothesis (Sec. 4's use of the previous estimate)."""
import math

import numpy as np

import oracle as orc
from paper_2210_14771_gb300 import synth


def _frame(seed=31, geometry="centred"):
    f, gt = synth.frame(seed, 0, 480, 640, geometry)
    return f, gt


def test_prior_without_support_changes_nothing():
    f, _ = _frame()
    p = orc.params(n_strips=16, cands_per_strip=2, n_hyps=64, seed=5)
    a = orc.estimate_tracked(f, 9, p, None)
    b = orc.estimate_tracked(f, 9, p, (20.0, 20.0, 5.0))   # no candidate near it
    assert a == b


def test_prior_alone_recovers_the_circle():
    """With no random hypotheses the result is the prior refined by the
    least-squares refits on its inliers: the true circle to about a pixel."""
    f, gt = _frame()
    p = orc.params(n_strips=16, cands_per_strip=2, n_hyps=0, seed=5)
    prior = (gt["cx"] + 2.0, gt["cy"] - 2.0, gt["r"] + 1.5)   # drifted by a few pixels
    r = orc.estimate_tracked(f, 9, p, prior)
    assert r["valid"] == 1
    assert math.hypot(r["cx"] - gt["cx"], r["cy"] - gt["cy"]) < 1.5 and abs(r["r"] - gt["r"]) < 1.5
    assert orc.estimate_tracked(f, 9, p, None)["valid"] == 0   # nothing without it


def test_better_prior_wins_and_ties_go_to_random_hypotheses():
    f, gt = _frame()
    p = orc.params(n_strips=16, cands_per_strip=2, n_hyps=8, seed=5)
    base = orc.estimate_tracked(f, 9, p, None)
    # the best random circle as prior: same support, a tie, lowest index wins
    same = orc.estimate_tracked(f, 9, p, (base["cx"], base["cy"], base["r"]))
    assert same["score"] == base["score"] and same["n_inliers"] == base["n_inliers"]
    good = orc.estimate_tracked(f, 9, p, (gt["cx"], gt["cy"], gt["r"]))
    assert good["score"] >= base["score"]


# ---- prior-guided scoring: the angle term points at the previous centre

def test_prior_centre2_rounding_and_clamping():
    """round(2 c), ties to even, clamped into the frame's doubled extent."""
    H, W = 480, 640
    assert orc.prior_centre2(10.25, 3.75, H, W) == (20, 8)       # 20.5 -> 20, 7.5 -> 8
    assert orc.prior_centre2(10.75, 3.25, H, W) == (22, 6)       # 21.5 -> 22, 6.5 -> 6
    assert orc.prior_centre2(319.5, 239.5, H, W) == (639, 479)   # the image centre
    assert orc.prior_centre2(-40.0, 1e4, H, W) == (0, 2 * (H - 1))
    assert orc.prior_centre2(5000.0, -0.2, H, W) == (2 * (W - 1), 0)


def test_image_centre_reduces_to_the_plain_candidates():
    p = orc.params(n_strips=16, cands_per_strip=4, n_hyps=64)
    for seed, geo in ((3, "centred"), (4, "clipped"), (5, "hard"), (6, "none")):
        f, _ = synth.frame(seed, 0, 480, 640, geo)
        a = orc.candidates(f, p)
        b = orc.candidates(f, p, (639, 479))
        assert all(np.array_equal(x, y) for x, y in zip(a, b)), (seed, geo)


def _step_frame(H=96, W=160, x_edge=100):
    """Bright content on the left, dark border on the right of a vertical step
    at x_edge (in the right half, whose preceding maximum is scanned from the
    dark right edge): every strip's strongest gradient is on the step and
    points in -x (dark -> bright)."""
    f = np.full((H, W, 3), 200, np.uint8)
    f[:, x_edge:] = 10
    return f


def test_centre_beyond_the_step_keeps_it_and_behind_it_drops_it():
    """The same step edge scores high when the centre lies on the side its
    gradient points to (angle 0) and is dropped by t_ps when the centre lies
    behind it (angle 180 degrees): a swapped axis or sign in the centre
    handling fails one of the two."""
    f = _step_frame()
    H, W = f.shape[:2]
    p = orc.params(n_strips=8, cands_per_strip=2, n_hyps=16, t_px=3.0)
    ahead = orc.candidates(f, p, (2 * 20, 2 * (H // 2)))     # centre left of the step
    behind = orc.candidates(f, p, (2 * 150, 2 * (H // 2)))   # centre right of the step
    xs_a, ys_a, ss_a = ahead
    assert len(xs_a) >= 6 and np.all(xs_a == 100)
    # the angle to the centre row y = 48 grows with |y - 48|: so does the penalty
    order = np.argsort(np.abs(ys_a.astype(int) - 48))
    assert np.all(np.diff(ss_a[order].astype(int)) <= 0)
    assert not np.any(np.isin(behind[0], (99, 100)))
    # a centre straight above the step: 90 degrees, s_theta = 1 - tanh(3), dropped
    side = orc.candidates(f, p, (2 * 100, 0))
    assert not np.any(np.isin(side[0], (99, 100)))
    # the image centre (79.5, 47.5) lies just left of the step: only the rows
    # near it keep their point
    plain = orc.candidates(f, p)
    assert 0 < len(plain[0]) < len(xs_a)


def test_tracked_estimate_with_prior_centre():
    """Without a prior, prior_centre changes nothing; with the true circle as
    prior on an off-centre frame, the candidates are those of the true centre."""
    f, gt = synth.frame(8, 0, 480, 640, "clipped")
    p = orc.params(n_strips=16, cands_per_strip=2, n_hyps=64, seed=3)
    assert orc.estimate_tracked(f, 1, p, None, True) == orc.estimate_tracked(f, 1, p, None)
    prior = (gt["cx"], gt["cy"], gt["r"])
    c2 = orc.prior_centre2(gt["cx"], gt["cy"], 480, 640)
    want = orc.fit(*orc.candidates(f, p, c2), 480, 640, 1, p, prior)
    assert orc.estimate_tracked(f, 1, p, prior, True) == want
