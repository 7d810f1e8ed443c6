"""Performance score of Eq. 2 over simulated time (Section V-A), from the runs' event logs.

This is host-side analysis of what the library records (ct_batch_events: each improvement of a
run's best with the simulated time at that evaluation); it is not a step of the search itself.
Definitions:

- baseline: valid configurations drawn uniformly without replacement; expected best after n
  draws E_n = sum_i f_(i) C(M-i, n-1) / C(M, n) over the sorted fitness values f_(1) <= ...;
  E_0 is the median.  A draw takes the mean evaluation time plus the per-proposal overhead.
- budget: the first n with E_n <= median - 0.95 (median - optimum), times the time per draw.
- a run evaluates its proposals one at a time in population order; its clock after the
  evaluation of index i in generation g: the evaluation time of every configuration evaluated
  so far (each once) plus (g * pop + i + 1) * overhead; its value at time t: its best after the
  last evaluation that ended by t, or the median while nothing valid has been evaluated.
- score at t: (E(t) - value(t)) / (E(t) - optimum), averaged over K times in (0, budget].
"""
from __future__ import annotations

import numpy as np

PENALTY = 1e20


class Baseline:
    """Random-search baseline of one space (fitness per valid rank, evaluation cost in us)."""

    def __init__(self, fit, cost_us, overhead_us: float = 0.0):
        self.f = np.sort(np.asarray(fit, np.float64))
        self.M = len(self.f)
        self.median = float(np.median(self.f))
        self.opt = float(self.f[0])
        self.per_draw = float(np.mean(np.asarray(cost_us, np.float64))) + overhead_us
        self._cache = {}

    def expected(self, n: int) -> float:
        """E_n.  Terms with C(M-i, n-1) / C(M, n) <= (n/M) e^-60 are dropped: that bound holds
        for i past M - (M-1) e^(-60/(n-1)) because each factor of the weight's product is at
        most (M-i)/(M-1)."""
        if n in self._cache:
            return self._cache[n]
        M = self.M
        if n == 0:
            v = self.median
        elif n == 1:
            v = float(self.f.mean())
        else:
            last = M - n + 1
            cut = int(np.ceil(M - (M - 1) * np.exp(-60.0 / (n - 1)))) + 1
            L = max(1, min(last, cut))
            # log w_i = log(n/M) + sum_{m<i} log(1 - (n-1)/(M-m))
            m = np.arange(1, L, dtype=np.float64)
            lw = np.log(n / M) + np.concatenate([[0.0], np.cumsum(np.log1p(-(n - 1) / (M - m)))])
            v = float(np.dot(self.f[:L], np.exp(lw)))
        self._cache[n] = v
        return v

    def budget(self):
        """(draws, time in us) of the budget rule; E_n is non-increasing, so bisect."""
        goal = self.median - 0.95 * (self.median - self.opt)
        lo, hi = 1, self.M
        while lo < hi:
            mid = (lo + hi) // 2
            if self.expected(mid) <= goal:
                hi = mid
            else:
                lo = mid + 1
        return lo, lo * self.per_draw


def run_scores(base: Baseline, events, pop, overhead_us: float = 0.0, K: int = 50):
    """Per-run scores (mean over the K sampled times) and per-time scores (mean over runs).
    events: per run, (generation, index, evaluation time, best) arrays of its improvements in
    evaluation order (ct_batch_events)."""
    n_star, B = base.budget()
    times = B * np.arange(1, K + 1) / K
    draws = np.minimum((times // base.per_draw).astype(np.int64), base.M)
    E = np.array([base.expected(int(n)) for n in draws])
    den = E - base.opt
    score = np.empty((len(events), K))
    for r, (gen, idx, clk, val) in enumerate(events):
        clock = np.asarray(clk, np.float64) + (np.asarray(gen, np.float64) * pop + np.asarray(idx, np.float64) + 1) * overhead_us
        v_ev = np.where(np.asarray(val, np.float64) < PENALTY, np.asarray(val, np.float64), base.median)
        e = np.searchsorted(clock, times, side="right") - 1          # last event by time t
        v = np.where(e >= 0, v_ev[np.maximum(e, 0)] if len(v_ev) else base.median, base.median)
        score[r] = np.where(den > 0, (E - v) / np.where(den > 0, den, 1.0), (v <= base.opt).astype(np.float64))
    return {"per_run": score.mean(axis=1), "per_time": score.mean(axis=0), "budget_us": B,
            "budget_draws": n_star, "times_us": times, "baseline": E}
