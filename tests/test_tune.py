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


class _Fake2(_Fake):
    def __init__(self, clock, cost, nu_of=lambda s, mf, tile: int(100 * s)):
        super().__init__(clock, None)
        self.cost2, self.nu_of2 = cost, nu_of
        self.tile = 64

    def set_schur_tile(self, edge):
        self.tile = edge

    def factor(self, s):
        self.clock.t += self.cost2(self.mf, self.tile)
        self.calls.append((self.mf, self.tile, s))

        class R:
            pass
        r = R()
        r.neg = self.nu_of2(s, self.mf, self.tile)
        return r


def test_joint_threshold_and_tile():
    clk = _Clock()
    cost = lambda mf, tile: 1.0 + abs(mf - 512) / 1000.0 + (0.1 if tile == 64 else 0.0)
    P = _Fake2(clk, cost)
    out = tune.tune_schur(P, [0.3], thresholds=(256, 512, 1024), tiles=(32, 64), clock=clk)
    assert out["best"] == (512, 32) and (P.mf, P.tile) == (512, 32)
    assert len(out["seconds"]) == 6 and len(P.calls) == 6 * 2
    clk2 = _Clock()
    P2 = _Fake2(clk2, lambda mf, tile: 1.0)
    assert tune.tune_schur(P2, [0.3], clock=clk2)["best"] == (1024, 64)      # ties: larger values
    P3 = _Fake2(_Clock(), lambda mf, tile: 1.0, nu_of=lambda s, mf, tile: 5 if tile == 32 else 6)
    with pytest.raises(RuntimeError):
        tune.tune_schur(P3, [0.3], clock=P3.clock)
