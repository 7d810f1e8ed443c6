"""The library's score (vectorised, truncated sums, bisection) against the oracle's plain one
on synthetic traces and seeded fitness tables."""
import numpy as np
import pytest

from oracle import score as OS
from paper_2606_28372_b300 import score as PS
from paper_2606_28372_b300 import workloads as W


@pytest.mark.parametrize("M,seed", [(7, 0), (732, 1), (20000, 2)])
def test_baseline_and_budget_match_the_oracle(M, seed):
    f = W.lognormal_table(M, seed=seed)
    c = W.eval_cost_table(f, seed=seed)
    b = PS.Baseline(f, c, overhead_us=250.0)
    for n in sorted({0, 1, 2, 3, M // 3, M - 1, M}):
        assert b.expected(n) == pytest.approx(OS.expected_best(f, n), rel=1e-10)
    n1, B1 = b.budget()
    n2, B2 = OS.budget(f, c, overhead_us=250.0)
    assert n1 == n2 and B1 == pytest.approx(B2, rel=1e-12)


def _events(f, R, P, seed):
    """Synthetic event logs: increasing (generation, index) positions and clocks, decreasing
    values; some runs start with penalised events (nothing valid yet)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(R):
        n = int(rng.integers(0, 30))
        pos = np.sort(rng.choice(60 * P, size=n, replace=False))
        clk = np.cumsum(rng.integers(0, 40, size=n)) * 1_600_000
        val = np.sort(rng.choice(f, size=n))[::-1].astype(np.float32)
        if r % 3 == 0 and n:
            val[: rng.integers(0, n)] = 1e20
        out.append((pos // P, pos % P, clk.astype(np.uint64), val))
    return out


@pytest.mark.parametrize("overhead", [0.0, 1000.0])
def test_scores_match_the_oracle(overhead):
    f = W.lognormal_table(5000, seed=3)
    c = W.eval_cost_table(f, seed=3)
    ev = _events(f, 12, 20, 4)
    a = PS.run_scores(PS.Baseline(f, c, overhead), ev, pop=20, overhead_us=overhead, K=40)
    e = OS.run_score(f, c, ev, pop=20, overhead_us=overhead, K=40)
    assert np.allclose(a["per_run"], e["per_run"], rtol=1e-9, atol=1e-9)
    assert np.allclose(a["per_time"], e["per_time"], rtol=1e-9, atol=1e-9)
    assert a["budget_draws"] == e["budget_draws"]
