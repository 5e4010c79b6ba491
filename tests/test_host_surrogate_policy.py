"""The hybrid solve's macro-step policy (the evaluation driver's copy of
fem_surrogate_solve's schedule): judged steps, the solver's spans after
failed judgements (doubling with each further consecutive failure, capped)
and the network's spans after passed ones.  Host logic only."""
import pytest

from paper_1005_3158_gb300.surrogate import MAX_BACKOFF, HybridPolicy


def _run(J, n, outcome):
    """Actions of n macro steps; outcome(k) -> passed for a judged step k."""
    pol = HybridPolicy(J)
    acts = []
    for k in range(n):
        a = pol.action(k)
        if a == "judge":
            pol.judged(k, outcome(k))
        acts.append(a)
    return acts


def _judged(acts):
    return [k for k, a in enumerate(acts) if a == "judge"]


def test_failures_double_the_span():
    acts = _run(8, 150, lambda k: False)
    assert _judged(acts) == [0, 8, 24, 56, 120]
    assert all(a == "solver" for a in acts if a != "judge")


def test_the_gpu_test_sequence():
    # fem_surrogate_solve with judge_every 2 over 20 macro steps and a
    # tolerance nothing meets judges steps 0, 2, 6 and 14 (4 failures)
    assert _judged(_run(2, 20, lambda k: False)) == [0, 2, 6, 14]


def test_passes_keep_the_cadence():
    acts = _run(8, 40, lambda k: True)
    assert _judged(acts) == [0, 8, 16, 24, 32]
    assert all(a == "network" for a in acts if a != "judge")


def test_a_pass_resets_the_backoff():
    outcomes = {0: False, 8: True, 16: False, 24: False}
    acts = _run(8, 48, lambda k: outcomes.get(k, False))
    assert _judged(acts) == [0, 8, 16, 24, 40]
    assert acts[1:8] == ["solver"] * 7          # after the failure at 0
    assert acts[9:16] == ["network"] * 7        # after the pass at 8
    assert acts[17:24] == ["solver"] * 7        # failure at 16: span 8 again
    assert acts[25:40] == ["solver"] * 15       # second failure in a row: 16


def test_span_is_capped():
    J = 1
    acts = _run(J, 1 + 2 + 4 + 8 + 16 + 32 + 64 + 64 + 64, lambda k: False)
    j = _judged(acts)
    spans = [b - a for a, b in zip(j, j[1:])]
    assert spans == [J << min(f, MAX_BACKOFF) for f in range(len(spans))]
    assert max(spans) == J << MAX_BACKOFF


@pytest.mark.parametrize("n", [1, 7, 30])
def test_no_judging(n):
    assert _run(0, n, lambda k: pytest.fail("judged")) == ["network"] * n
