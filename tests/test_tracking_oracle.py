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
