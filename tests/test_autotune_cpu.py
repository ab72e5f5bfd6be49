"""The leaf-size autotuner's choice rule (host logic, no GPU): the fastest
candidate wins, but the default leaf size stays unless another one is faster
by more than the tie margin."""
from paper_2112_06188_gb300 import autotune


def test_choose_fastest_beyond_tie():
    assert autotune.choose({8: 9.0, 16: 10.0, 32: 11.0}) == 8
    assert autotune.choose({8: 10.4, 16: 10.0, 32: 9.8}) == 32


def test_choose_keeps_default_within_tie():
    d = autotune.DEFAULT
    ms = {8: 10.0 * (1 - autotune.TIE / 2), d: 10.0, 32: 10.3}
    assert autotune.choose(ms) == d
    assert autotune.choose({d: 5.0}) == d


def test_choose_without_default():
    assert autotune.choose({8: 10.0, 32: 9.0}) == 32
