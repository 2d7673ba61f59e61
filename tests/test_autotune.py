"""Selection logic of the launch autotuner (host only, CPU)."""
import pytest

from paper_2501_18054_gb300 import autotune as A


def test_candidates_respect_capacity_and_refresh():
    c = A.candidates(4096, 152, 64)
    assert c and all(x.ctas == 152 // x.runs for x in c)
    assert all(4096 <= 256 * x.ctas for x in c)  # at most 256 pixels per CTA
    assert {x.runs for x in c} == {1, 2, 3, 4}
    assert all(64 % x.delay_r == 0 for x in c)
    # eight runs: 19 CTAs of 216 pixels (224 rounded); R = 64 leaves (64 + 8) x 224 x 8 = 129 KB
    eight = A.candidates(4096, 152, 64, runs_options=(8,), delay_options=(64, 128))
    assert {x.delay_r for x in eight} == {64}  # R = 128 would need 243 KB
    # ten runs: 15 CTAs of 274 pixels, above 256 per CTA
    assert not A.candidates(4096, 152, 64, runs_options=(10,))
    assert not A.candidates(4096, 152, 48, delay_options=(32,))  # 48 is not a multiple of 32
    assert len(A.candidates(100, 152, 64, runs_options=(1, 2, 4, 8), delay_options=(16, 32, 64))) == 4 * 3 * 2


def _fake(speed, bad=()):
    """A deterministic stand-in for timed trials: evals/s from a model, and
    accuracy failures for the listed candidates."""
    calls = []

    def measure(cand, steps):
        calls.append((cand, steps))
        v = speed(cand) * (1.0 + 0.001 * steps)
        accurate = cand not in bad
        return A.Trial(cand, steps, v, 1e-7 if accurate else 3e-4, True)

    return measure, calls


def test_tune_picks_the_fastest_accurate_configuration():
    cands = A.candidates(4096, 152, 64)

    def speed(c):  # more runs help, the tensor-core fold helps, R = 32 slightly better
        return 1e6 * c.runs * (1.3 if c.tensor_fold else 1.0) * (1.02 if c.delay_r == 32 else 1.0)

    best_model = max(cands, key=speed)
    measure, calls = _fake(speed, bad={best_model})  # the fastest one misses the accuracy bar
    log = []
    win, trials = A.tune(cands, measure, log=log)
    assert win.cand != best_model
    assert win.cand == max((c for c in cands if c != best_model), key=speed)
    assert win.steps == 3
    # every candidate was timed once briefly, a third of the accurate ones again
    assert sum(1 for c, s in calls if s == 1) == len(cands)
    n_good = len(cands) - 1
    assert sum(1 for c, s in calls if s == 3) == -(-n_good // 3)
    assert len(log) == len(trials)


def test_select_rejects_inaccurate_and_failed_trials():
    c1, c2 = A.Candidate(4, 38, 64, 1), A.Candidate(2, 76, 64, 1)
    t_fast_bad = A.Trial(c1, 3, 9e6, 2e-4, True)
    t_fast_diff = A.Trial(c1, 3, 9e6, 1e-8, False)
    t_fast_fail = A.Trial(c1, 3, 9e6, 1e-8, True, ok=False)
    t_slow = A.Trial(c2, 3, 5e6, 1e-6, True)
    assert A.select([t_fast_bad, t_fast_diff, t_fast_fail, t_slow]).cand == c2
    with pytest.raises(ValueError):
        A.select([t_fast_bad, t_fast_diff])


def test_ties_prefer_fewer_runs_then_smaller_delay():
    a, b, c = A.Candidate(4, 38, 64, 1), A.Candidate(2, 76, 64, 1), A.Candidate(2, 76, 32, 1)
    ts = [A.Trial(x, 3, 5e6, 1e-7, True) for x in (a, b, c)]
    assert A.select(ts).cand == c
