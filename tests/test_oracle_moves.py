"""Pins of the oracle's PSO and Firefly moves and of DE's selection (Sections IV-B and IV-C).

The paper prints no trace of these optimizers, so each test isolates one term of the update at
hyper-parameters where the others vanish and checks the direction and size of the move it makes,
or checks Algorithm 1's acceptance rule against the trace of whole runs.  Each is chosen so that a
plausible mistake fails it: a sign error in p - x or g - x, c1 and c2 swapped, the two PSO draws
swapped, a lost velocity carry, a firefly that moves away from a brighter one, a wrong beta
(exp of +gamma r^2, r instead of r^2), a wrong noise term, and a DE that rejects good trials,
accepts members already present, accepts a duplicate of an earlier trial or uses < for <=.
"""
import numpy as np
import pytest

from paper_2606_28372_b300 import workloads as W

PSO_R, FA_ALPHA, PSO_VEL = 4, 5, 13
CROSS = 3
f32 = np.float32


@pytest.fixture(scope="module")
def medium(oracle_mod):
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    return sd, sp, keys, W.smooth_table(sd, oracle_mod.unpack(sp, keys), seed=0)


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    sd = W.tiny_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    return sd, sp, keys, W.lognormal_table(len(keys), seed=0)


def _eps(sp):
    return f32(1.0) / f32(int(sp.r.max()) - 1)


def _u01(O, seed, i, g, purpose, t):
    return f32((O.rng_word(seed, i, g, purpose, t) >> 8) * 2.0 ** -24)


def _clip(x):
    return np.minimum(np.maximum(x, f32(0)), f32(1))


def test_pso_initial_positions_are_the_grid_points(oracle_mod, medium):
    sd, sp, keys, table = medium
    T = oracle_mod.run("pso", sp, keys, table, pop=16, gens=1, seed=2)
    idx = oracle_mod.unpack(sp, T["cand"][0]).astype(np.float32)
    assert np.array_equal(T["pos"][0], idx * _eps(sp))


def test_pso_inertia_only_carries_the_initial_velocity(oracle_mod, medium):
    """w = 1, c1 = c2 = 0: the velocity stays v0 = (2u - 1) eps, and every coordinate moves by
    exactly v0 per generation until it is clipped to [0, 1]."""
    sd, sp, keys, table = medium
    P, seed, G = 16, 3, 8
    T = oracle_mod.run("pso", sp, keys, table, pop=P, gens=G, seed=seed, pso_w=1.0, pso_c1=0.0, pso_c2=0.0)
    eps, n = _eps(sp), sp.n
    v0 = np.array([[(f32(2) * _u01(oracle_mod, seed, i, 0, PSO_VEL, j) - f32(1)) * eps for j in range(n)]
                   for i in range(P)], dtype=np.float32)
    assert (v0 > 0).any() and (v0 < 0).any()
    x = T["pos"][0].copy()
    for g in range(1, G + 1):
        x = _clip((x + v0).astype(np.float32))
        assert np.array_equal(T["pos"][g], x), g
    assert ((x == 0) | (x == 1)).any()          # some coordinates reached a bound and stayed there


def test_pso_cognitive_term_pulls_toward_personal_best(oracle_mod, medium):
    """w = 1, c1 = 3, c2 = 0.  Generation 1 moves by v0 (pbest = x0).  A particle that did not
    improve keeps pbest = x0, so in generation 2 its velocity changes by c1 r1 (x0 - x1), with
    r1 the first of the two PSO draws of that coordinate: back toward x0, scaled by r1.  A
    particle that improved has pbest = x1 and keeps its velocity."""
    sd, sp, keys, table = medium
    P, seed = 64, 7
    T = oracle_mod.run("pso", sp, keys, table, pop=P, gens=2, seed=seed, pso_w=1.0, pso_c1=3.0, pso_c2=0.0)
    x0, x1, x2 = (T["pos"][g].astype(np.float64) for g in range(3))
    f0, f1 = T["fit"][0], T["fit"][1]
    checked = kept = 0
    for i in range(P):
        for j in range(sp.n):
            if not (0 < x1[i, j] < 1 and 0 < x2[i, j] < 1 and x1[i, j] != x0[i, j]):
                continue
            dv = (x2[i, j] - x1[i, j]) - (x1[i, j] - x0[i, j])
            if f1[i] < f0[i]:                                   # pbest moved to x1: no pull
                assert abs(dv) < 1e-6
                kept += 1
                continue
            r1 = float(_u01(oracle_mod, seed, i, 2, PSO_R, 2 * j))
            want = 3.0 * r1 * (x0[i, j] - x1[i, j])
            assert dv * (x0[i, j] - x1[i, j]) >= 0               # toward pbest, never away
            assert abs(dv - want) < 1e-6, (i, j, dv, want)
            checked += 1
    assert checked >= 20 and kept >= 1


def test_pso_social_term_pulls_toward_global_best(oracle_mod, medium):
    """w = 0, c1 = 0, c2 = 0.5: in generation 1 every particle moves toward gbest, the position
    of the first particle with the lowest fitness, by c2 r2 (g - x) with r2 the second PSO draw;
    it stays between x and gbest, and gbest's own particle does not move."""
    sd, sp, keys, table = medium
    P, seed = 32, 5
    T = oracle_mod.run("pso", sp, keys, table, pop=P, gens=1, seed=seed, pso_w=0.0, pso_c1=0.0, pso_c2=0.5)
    x0, x1 = T["pos"][0].astype(np.float64), T["pos"][1].astype(np.float64)
    b = int(np.argmin(T["fit"][0]))
    gb = x0[b]
    assert np.array_equal(x1[b], x0[b])
    moved = 0
    for i in range(P):
        for j in range(sp.n):
            d = gb[j] - x0[i, j]
            step = x1[i, j] - x0[i, j]
            assert step * d >= 0 and abs(step) <= 0.5 * abs(d) + 1e-7
            r2 = float(_u01(oracle_mod, seed, i, 1, PSO_R, 2 * j + 1))
            assert abs(step - 0.5 * r2 * d) < 1e-6, (i, j)
            moved += d != 0
    assert moved >= 20


def _two_fireflies(oracle_mod, medium, seed, **prm):
    sd, sp, keys, table = medium
    T = oracle_mod.run("firefly", sp, keys, table, pop=2, gens=1, seed=seed, **prm)
    f = T["fit"][0]
    assert f[0] != f[1]
    bright, dim = (0, 1) if f[0] < f[1] else (1, 0)
    x0 = T["pos"][0].astype(np.float64)
    x1 = T["pos"][1].astype(np.float64)
    assert np.array_equal(x1[bright], x0[bright])            # nothing brighter: it stays
    assert not np.array_equal(x0[dim], x0[bright])
    return sp, x0[dim], x0[bright], x1[dim], bright


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_firefly_full_attraction_lands_on_the_brighter(oracle_mod, medium, seed):
    """beta0 = 1, gamma = 0, alpha = 0: beta = 1, so the dimmer firefly lands on the brighter."""
    _, y, xb, y1, _ = _two_fireflies(oracle_mod, medium, seed, fa_beta0=1.0, fa_gamma=0.0, fa_alpha=0.0)
    assert np.abs(y1 - xb).max() < 1e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_firefly_half_attraction_lands_on_the_midpoint(oracle_mod, medium, seed):
    _, y, xb, y1, _ = _two_fireflies(oracle_mod, medium, seed, fa_beta0=0.5, fa_gamma=0.0, fa_alpha=0.0)
    assert np.abs(y1 - (y + xb) / 2).max() < 1e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_firefly_attraction_decays_with_squared_distance(oracle_mod, medium, seed):
    """beta0 = 1, gamma = 1, alpha = 0: the step is exp(-r^2) of the way to the brighter one,
    r^2 the squared Euclidean distance between the two positions."""
    _, y, xb, y1, _ = _two_fireflies(oracle_mod, medium, seed, fa_beta0=1.0, fa_gamma=1.0, fa_alpha=0.0)
    r2 = float(np.sum((y - xb) ** 2))
    beta = np.exp(-r2)
    assert 0 < beta < 1
    assert np.abs(y1 - (y + beta * (xb - y))).max() < 2e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_firefly_without_attraction_moves_by_noise_only(oracle_mod, medium, seed):
    """beta0 = 0, alpha = 0.2: the dimmer firefly moves by alpha (u - 0.5) per coordinate, u the
    FA_ALPHA draw of (brighter index, coordinate); so by at most alpha / 2."""
    sp, y, xb, y1, bright = _two_fireflies(oracle_mod, medium, seed, fa_beta0=0.0, fa_gamma=1.0, fa_alpha=0.2)
    dim = 1 - bright
    n = sp.n
    u = np.array([_u01(oracle_mod, seed, dim, 1, FA_ALPHA, bright * n + d) for d in range(n)], dtype=np.float64)
    want = np.clip(y + 0.2 * (u - 0.5), 0.0, 1.0)
    assert np.abs(y1 - want).max() < 1e-6
    assert np.abs(y1 - y).max() <= 0.1 + 1e-6


def _check_de_selection(T, P, G):
    """Algorithm 1's selection replayed on the trace: in ascending i, trial u_i replaces x_i iff
    f(u_i) <= f(x_i), u_i is not in the generation's starting population, and no earlier trial of
    the generation with the same key was accepted; two generations without an acceptance re-draw
    the population in the next one.  Returns how often each clause decided."""
    seen = dict(accepted=0, worse=0, in_x=0, duplicate=0, ties=0, reinit=0)
    stag, pending = 0, False
    for g in range(1, G + 1):
        if pending:
            assert np.array_equal(T["popk"][g], T["evalk"][g]) and np.array_equal(T["popf"][g], T["fit"][g])
            pending, stag = False, 0
            seen["reinit"] += 1
            continue
        X0, F0 = T["popk"][g - 1], T["popf"][g - 1]
        U, FU = T["evalk"][g], T["fit"][g]
        start = set(int(k) for k in X0)
        X1, F1 = X0.copy(), F0.copy()
        taken = set()
        acc = 0
        for i in range(P):
            u = int(U[i])
            if not FU[i] <= F0[i]:
                seen["worse"] += 1
            elif u in start:
                seen["in_x"] += 1
            elif u in taken:
                seen["duplicate"] += 1
            else:
                seen["ties"] += bool(FU[i] == F0[i])
                X1[i], F1[i] = U[i], FU[i]
                taken.add(u)
                acc += 1
        assert np.array_equal(T["popk"][g], X1), g
        assert np.array_equal(T["popf"][g], F1), g
        seen["accepted"] += acc
        stag = 0 if acc else stag + 1
        if stag >= 2:
            pending, stag = True, 0
    return seen


def test_de_selection_follows_algorithm_1(oracle_mod, tiny):
    """On the tiny space with a table of four distinct values (so that equal fitness is common
    and the <= of Algorithm 1 matters), small populations (duplicate trials) and several seeds,
    every generation's population is the one the acceptance rule gives, and every clause of the
    rule decides some trial."""
    sd, sp, keys, table = tiny
    q = np.quantile(table, [0.25, 0.5, 0.75])
    coarse = np.digitize(table, q).astype(np.float32) + 1.0
    total = dict(accepted=0, worse=0, in_x=0, duplicate=0, ties=0, reinit=0)
    for seed in range(6):
        for P in (8, 20):
            T = oracle_mod.run("de", sp, keys, coarse, pop=P, gens=60, seed=seed)
            for k, v in _check_de_selection(T, P, 60).items():
                total[k] += v
    assert all(v > 0 for v in total.values()), total


def test_de_selection_medium_lognormal(oracle_mod, medium):
    sd, sp, keys, table = medium
    T = oracle_mod.run("de", sp, keys, table, pop=32, gens=40, seed=11)
    seen = _check_de_selection(T, 32, 40)
    assert seen["accepted"] > 0 and seen["worse"] > 0


@pytest.mark.parametrize("seed", [13, 14, 15])
def test_de_best_update_and_f0_cr0_trials(oracle_mod, tiny, seed):
    """F = 0, CR = 0: each trial is x_i with gene j_rand taken from best.  Replaying best by
    Algorithm 1's rule (accepted trials scanned in ascending i, best <- u if f(u) <= f(best); the
    initial and re-drawn populations scanned the same way) predicts every generation's trials.
    A table of four distinct values makes equal fitness common, so <= against < matters."""
    sd, sp, keys, table = tiny
    q = np.quantile(table, [0.25, 0.5, 0.75])
    coarse = np.digitize(table, q).astype(np.float32) + 1.0
    P, G = 20, 40
    T = oracle_mod.run("de", sp, keys, coarse, pop=P, gens=G, seed=seed, de_F=0.0, de_CR=0.0)

    def scan(rows, g, best):
        for i in rows:
            if T["popf"][g][i] <= best[1]:
                best = (T["popk"][g][i], T["popf"][g][i])
        return best

    best = scan(range(1, P), 0, (T["popk"][0][0], T["popf"][0][0]))
    stag, pending, checked, moved_best = 0, False, 0, 0
    for g in range(1, G + 1):
        if pending:                                      # re-drawn population; best persists
            best = scan(range(P), g, best)
            pending, stag = False, 0
            continue
        ib = oracle_mod.unpack(sp, [best[0]])[0]
        X = oracle_mod.unpack(sp, T["popk"][g - 1])
        got = oracle_mod.unpack(sp, T["cand"][g])
        for i in range(P):
            jr = (oracle_mod.rng_word(seed, i, g, CROSS, 0) * sp.n) >> 32
            want = X[i].copy()
            want[jr] = ib[jr]
            assert np.array_equal(got[i], want), (g, i)
            checked += 1
        acc = [i for i in range(P) if T["popk"][g][i] != T["popk"][g - 1][i]]
        before = best
        best = scan(acc, g, best)
        moved_best += best[0] != before[0] and best[1] == before[1]
        stag = 0 if acc else stag + 1
        if stag >= 2:
            pending, stag = True, 0
    assert checked >= P * G // 2
