"""The batched workload's problem draws: sizes, wavenumber range, face rules, determinism."""
import helm6_inputs as inputs


def test_batch_problem_draws():
    probs = inputs.batch_problems(0, 64)
    assert len(probs) == 64
    assert probs == inputs.batch_problems(0, 64)
    assert probs != inputs.batch_problems(1, 64)
    for p in probs:
        assert p["n"] in inputs.BATCH_SIZES
        assert 5.0 <= p["k"].real <= 60.0 and abs(p["k"].imag - 0.01 * p["k"].real) < 1e-12
        assert all(c in "DN" for c in p["faces"][:4]) and all(c in "DNS" for c in p["faces"][4:])
    # every size class, and both Sommerfeld-like and other z faces, occur in 64 draws
    assert {p["n"] for p in probs} == set(inputs.BATCH_SIZES)
    assert any("S" in p["faces"] for p in probs) and any("S" not in p["faces"] for p in probs)
