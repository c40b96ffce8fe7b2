"""Host logic of the parameter autotuner (no GPU): the choice rule."""
from paper_2210_14771_gb300.tune import Trial, choose


def T(N, NH, ms, nh, miss):
    return Trial(N, 2, NH, ms, nh, miss)


def test_choose_fastest_not_less_accurate():
    ref = T(32, 1024, 1.0, 5.0, 10.0)
    trials = [ref, T(16, 512, 0.3, 7.0, 10.0), T(16, 1024, 0.5, 5.0, 10.0),
              T(64, 4096, 3.0, 2.0, 5.0), T(32, 512, 0.6, 4.9, 10.0)]
    assert choose(trials, ref) is trials[2]      # 0.5 ms, as accurate as the reference


def test_choose_keeps_reference_when_nothing_qualifies():
    ref = T(32, 1024, 1.0, 5.0, 10.0)
    trials = [ref, T(16, 512, 0.3, 7.0, 10.0), T(64, 512, 0.4, 4.0, 12.0)]
    assert choose(trials, ref) is ref


def test_choose_ties_in_time_go_to_accuracy():
    ref = T(32, 1024, 1.0, 5.0, 10.0)
    a, b = T(16, 512, 0.5, 4.0, 10.0), T(16, 1024, 0.5, 3.0, 10.0)
    assert choose([ref, a, b], ref) is b


def P(N, NH, ms, nh_frames):
    import numpy as np
    nh = np.asarray(nh_frames, float)
    return Trial(N, 2, NH, ms, float(nh.mean()), float((nh > 15).mean() * 100), {}, nh)


def test_paired_rule_ignores_frame_noise_but_not_real_loss():
    """Per-frame NH: a trial 0.05 px worse on average with a spread of 0.5 px
    is within noise (no worse); one uniformly 1 px worse is worse; one that
    adds a miss is worse whatever its mean."""
    import numpy as np
    rng = np.random.default_rng(0)
    base = rng.uniform(1.0, 6.0, 64)
    ref = P(32, 1024, 1.0, base)
    noisy = P(16, 512, 0.3, base + 0.05 + rng.normal(0.0, 0.5, 64))
    worse = P(16, 1024, 0.4, base + 1.0)
    miss = base.copy()
    miss[3] = 40.0
    missed = P(16, 4096, 0.5, miss - 0.3)
    from paper_2210_14771_gb300.tune import no_worse
    assert no_worse(noisy, ref) and not no_worse(worse, ref) and not no_worse(missed, ref)
    assert choose([ref, noisy, worse, missed], ref) is noisy


def test_calibration_subset_takes_classes_in_turn():
    from paper_2210_14771_gb300.tune import calibration_subset
    gts = [{"kind": k} for k in ["clipped"] * 10 + ["full"] * 3 + ["none"] * 2]
    sub = calibration_subset(gts, 8)
    kinds = [gts[i]["kind"] for i in sub]
    assert len(sub) == 8 and kinds.count("full") == 3 and kinds.count("none") == 2
    assert sub == sorted(sub)
