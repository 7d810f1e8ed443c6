"""CPU oracle of the performance score — TEST INFRASTRUCTURE ONLY (tests, the benchmark's CPU leg).

Follows Section V-A: the performance score of Eq. 2 over simulated time, against a calculated
random-search baseline, with the budget rule (the time the baseline needs to close 95 % of the
gap between the median and the optimum of the space).  The paper gives the definition in words
and defers the details to the methodology it cites; the readings taken here:

- the baseline draws valid configurations uniformly without replacement; its expected best
  after n draws is the mean of the minimum over all n-subsets of the valid fitness values;
  before the first draw it stands at the median;
- every draw of the baseline takes the mean evaluation time of the space plus the per-proposal
  overhead, so its value at time t is the expectation after floor(t / that) draws;
- a run evaluates its proposals one at a time, in population order within a generation; its
  simulated clock after an evaluation is the evaluation time of every configuration evaluated
  so far (each once) plus the overhead of every proposal made so far; its value at time t is
  its best fitness after the last evaluation that ended by t, or the median while it has
  evaluated nothing valid;
- the score of a run at t is (baseline(t) - value(t)) / (baseline(t) - optimum): 0 on the
  baseline, 1 at the optimum; it is averaged over K evenly spaced times in (0, budget] and
  over runs (and Eq. 2 averages that over spaces).

Plain fp64 arithmetic, no truncation and no vectorised search: small spaces only.
"""
from __future__ import annotations

import numpy as np


def expected_best(fit, n):
    """Mean of the minimum of n values drawn without replacement from ``fit`` (n = 0: median).

    P(the i-th smallest value is the minimum) = C(M-i, n-1) / C(M, n); the weights follow from
    w_1 = n / M and w_{i+1} / w_i = (M - i - n + 1) / (M - i)."""
    f = np.sort(np.asarray(fit, np.float64))
    M = len(f)
    if n == 0:
        return float(np.median(f))
    if not 1 <= n <= M:
        raise ValueError("n outside 0..M")
    L = M - n + 1                                   # only the L smallest can be the minimum
    i = np.arange(1, L, dtype=np.float64)           # ratios for i = 1 .. L-1
    ratio = (M - i - n + 1) / (M - i)
    w = np.concatenate([[n / M], (n / M) * np.cumprod(ratio)])
    return float(np.dot(f[:L], w))


def budget(fit, cost_us, overhead_us=0.0):
    """(draws, time): the first n with expected_best(n) <= median - 0.95 (median - optimum),
    and n times the baseline's time per draw."""
    f = np.asarray(fit, np.float64)
    med, opt = float(np.median(f)), float(f.min())
    goal = med - 0.95 * (med - opt)
    per = float(np.mean(np.asarray(cost_us, np.float64))) + overhead_us
    n = 1
    while expected_best(f, n) > goal:
        n += 1
    return n, n * per


def run_score(fit, cost_us, events, pop, overhead_us=0.0, K=50, penalty=1e20):
    """Score of each run from its event log and the per-time-point scores averaged over runs.

    ``events`` holds, per run, the improvements of its best in evaluation order as four
    sequences: generation, population index, simulated evaluation time after that evaluation
    (each configuration charged once), new best.  The clock of an event adds the overhead of
    every proposal up to and including it: (generation * pop + index + 1) * overhead."""
    f = np.asarray(fit, np.float64)
    med, opt = float(np.median(f)), float(f.min())
    nstar, B = budget(f, cost_us, overhead_us)
    per = float(np.mean(np.asarray(cost_us, np.float64))) + overhead_us
    times = [B * k / K for k in range(1, K + 1)]
    base = [expected_best(f, min(int(t // per), len(f))) for t in times]
    R = len(events)
    scores = np.zeros((R, K))
    for r in range(R):
        gen, idx, clk, val = events[r]
        for k, t in enumerate(times):
            value = med
            for e in range(len(gen)):
                clock = float(clk[e]) + (int(gen[e]) * pop + int(idx[e]) + 1) * overhead_us
                if clock > t:
                    break
                value = float(val[e]) if float(val[e]) < penalty else med
            den = base[k] - opt
            if den > 0:
                scores[r, k] = (base[k] - value) / den
            else:
                scores[r, k] = 1.0 if value <= opt else 0.0
    return {"per_run": scores.mean(axis=1), "per_time": scores.mean(axis=0), "budget_us": B,
            "budget_draws": nstar, "times_us": np.array(times), "baseline": np.array(base)}
