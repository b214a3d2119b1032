"""The threshold autotuner's host logic, driven through a stand-in problem whose factorization
time is a known function of the threshold (no GPU): it keeps the fastest candidate, leaves it set,
breaks ties toward the larger threshold, and rejects counts that change with the threshold."""
import pytest

from paper_1710_05134_gb300 import tune


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class _Fake:
    def __init__(self, clock, cost, nu_of=lambda s, mf: int(100 * s)):
        self.clock, self.cost, self.nu_of = clock, cost, nu_of
        self.mf = None
        self.calls = []

    def set_schur_mode(self, emulated, min_front):
        assert emulated
        self.mf = min_front

    def factor(self, s):
        self.clock.t += self.cost(self.mf)
        self.calls.append((self.mf, s))

        class R:
            pass
        r = R()
        r.neg = self.nu_of(s, self.mf)
        return r


def test_keeps_the_fastest_threshold():
    clk = _Clock()
    P = _Fake(clk, lambda mf: 1.0 + ((mf - 600) / 1000.0) ** 2)        # fastest near 600
    out = tune.tune_min_front(P, [0.3, 0.4], candidates=(256, 512, 768, 1024), reps=2, clock=clk)
    assert out["best"] == 512 and P.mf == 512
    assert all(abs(out["seconds"][m] - (1.0 + ((m - 600) / 1000.0) ** 2)) < 1e-12 for m in (256, 512, 768, 1024))
    assert out["nu"] == [30, 40, 30, 40]
    # one untimed factorization per candidate plus reps x shifts timed ones
    assert len(P.calls) == 4 * (1 + 2 * 2)


def test_ties_go_to_the_larger_threshold():
    clk = _Clock()
    P = _Fake(clk, lambda mf: 2.0)
    assert tune.tune_min_front(P, [0.1], candidates=(512, 1024, 768), clock=clk)["best"] == 1024


def test_changing_counts_are_rejected():
    clk = _Clock()
    P = _Fake(clk, lambda mf: 1.0, nu_of=lambda s, mf: 7 if mf < 1000 else 8)
    with pytest.raises(RuntimeError):
        tune.tune_min_front(P, [0.1], candidates=(512, 1024), clock=clk)
    with pytest.raises(ValueError):
        tune.tune_min_front(P, [], clock=clk)
