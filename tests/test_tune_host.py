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
