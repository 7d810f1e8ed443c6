"""Pins of the oracle's performance score (Eq. 2 over simulated time, Section V-A): the baseline
against brute force over all subsets and its closed-form ends, the budget crossing, and the
score's fixed points (0 on the baseline, 1 at the optimum, negative when nothing is found)."""
import itertools

import numpy as np
import pytest

from oracle import score as S


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_expected_best_is_the_mean_minimum_over_all_subsets(seed):
    rng = np.random.default_rng(seed)
    f = rng.lognormal(size=8)
    f[3] = f[5]                                     # a tie
    for n in range(1, 9):
        brute = np.mean([min(c) for c in itertools.combinations(f, n)])
        assert S.expected_best(f, n) == pytest.approx(brute, rel=1e-12)
    assert S.expected_best(f, 0) == np.median(f)


def test_expected_best_ends():
    f = np.random.default_rng(3).lognormal(size=5000)
    assert S.expected_best(f, 1) == pytest.approx(f.mean(), rel=1e-12)
    assert S.expected_best(f, len(f)) == pytest.approx(f.min(), rel=1e-12)
    e = [S.expected_best(f, n) for n in (1, 2, 5, 50, 500)]
    assert all(a > b for a, b in zip(e, e[1:]))


def test_budget_is_the_first_crossing():
    rng = np.random.default_rng(4)
    f = rng.lognormal(size=3000)
    c = rng.integers(1000, 3000, size=3000)
    n, B = S.budget(f, c, overhead_us=500.0)
    goal = np.median(f) - 0.95 * (np.median(f) - f.min())
    assert S.expected_best(f, n) <= goal < S.expected_best(f, n - 1)
    assert B == pytest.approx(n * (c.mean() + 500.0))


def _ev(gen, idx, clk, val):
    return (np.asarray(gen), np.asarray(idx), np.asarray(clk, np.float64), np.asarray(val, np.float64))


def test_score_fixed_points():
    rng = np.random.default_rng(5)
    f = rng.lognormal(size=2000)
    c = np.full(2000, 1000)
    P, K = 4, 20
    out = S.run_score(f, c, [_ev([0], [0], [0], [f.max()])], pop=P, K=K)
    times, base = out["times_us"], out["baseline"]
    # a run that holds the optimum from the first instant scores 1
    r1 = S.run_score(f, c, [_ev([0], [0], [0], [f.min()])], pop=P, K=K)
    assert r1["per_run"][0] == pytest.approx(1.0)
    # a run whose value is the baseline's at every sampled time scores 0
    z = np.zeros(K, int)
    r0 = S.run_score(f, c, [_ev(z, z, times - 0.5, base)], pop=P, K=K)
    assert r0["per_run"][0] == pytest.approx(0.0, abs=1e-12)
    # a run that never evaluates a valid configuration scores below 0
    rn = S.run_score(f, c, [_ev([0], [0], [0], [1e20])], pop=P, K=K)
    assert rn["per_run"][0] < 0
    # an event counts from its own evaluation on, proposal overheads included
    o = 10.0
    ref = S.run_score(f, c, [_ev([], [], [], [])], pop=P, overhead_us=o, K=K)
    times, base = ref["times_us"], ref["baseline"]
    assert o <= times[0]
    ev = _ev([0, 1], [0, P - 1], [0, times[4] - 2 * P * o], [np.median(f), f.min()])
    tr = S.run_score(f, c, [ev], pop=P, overhead_us=o, K=K)     # the second ends exactly at the 5th time
    head = sum((b - np.median(f)) / (b - f.min()) for b in base[:4])
    assert tr["per_run"][0] == pytest.approx((head + (K - 4)) / K, rel=1e-12)


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
@pytest.mark.parametrize("aware", [1, 0])
def test_run_clock_is_the_cost_of_each_configuration_evaluated_once(oracle_mod, kind, aware):
    from paper_2606_28372_b300 import workloads as W
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    table = W.smooth_table(sd, oracle_mod.unpack(sp, keys), seed=0)
    cost = W.eval_cost_table(table, seed=1)
    T = oracle_mod.run(kind, sp, keys, table, pop=24, gens=15, seed=2, cost=cost, constraint_aware=aware)
    rk = oracle_mod.lookup(keys, T["evalk"].ravel()).reshape(T["evalk"].shape)
    for g in range(16):
        seen = np.unique(rk[: g + 1][rk[: g + 1] >= 0])
        assert int(T["cost"][g]) == int(cost[seen].astype(np.uint64).sum())
    T0 = oracle_mod.run(kind, sp, keys, table, pop=24, gens=15, seed=2, constraint_aware=aware)
    assert (T0["cost"] == 0).all()
    for f in ("evalk", "best_fit", "n_unique"):      # the clock does not steer the run
        assert np.array_equal(T0[f], T[f])


@pytest.mark.parametrize("kind", ["de", "ga", "pso"])
@pytest.mark.parametrize("aware", [1, 0])
def test_event_log_is_the_running_best_in_evaluation_order(oracle_mod, kind, aware):
    """Events = strict improvements of the running minimum over the evaluated fitness, read
    generation by generation in population order; each carries the running sum of the costs of
    first evaluations up to it."""
    from paper_2606_28372_b300 import workloads as W
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    table = W.smooth_table(sd, oracle_mod.unpack(sp, keys), seed=0)
    cost = W.eval_cost_table(table, seed=1)
    T = oracle_mod.run(kind, sp, keys, table, pop=24, gens=20, seed=6, cost=cost, constraint_aware=aware)
    fit, evk = T["fit"].ravel(), T["evalk"].ravel()
    rk = oracle_mod.lookup(keys, evk)
    seen, clock, best = set(), 0, np.inf
    exp = []
    for e in range(len(fit)):
        if rk[e] >= 0 and rk[e] not in seen:
            seen.add(rk[e])
            clock += int(cost[rk[e]])
        if fit[e] < best:
            best = fit[e]
            exp.append((e // 24, e % 24, clock, fit[e]))
    got = list(zip(T["ev_gen"], T["ev_idx"], T["ev_clock"], T["ev_fit"]))
    assert [(int(a), int(b), int(c), np.float32(d)) for a, b, c, d in got] == \
        [(int(a), int(b), int(c), np.float32(d)) for a, b, c, d in exp]
