"""Pins of the oracle's DE and GA operator variants (Section IV-B: rand/best with up to five
random vectors, current-to-best, rand-to-best, binomial or exponential crossover; Section IV-D:
single-point, two-point, uniform and disruptive uniform crossover).

DE: with a population of partners + 1 every other member is a partner, so the trial must be the
textbook formula (evaluated in float32 numpy) for one ordering of the other members.  GA: every
child pair must come from two members of the previous population by the variant's structure."""
import itertools

import numpy as np
import pytest

from paper_2606_28372_b300 import workloads as W

PARTNERS = {"best1": 2, "rand1": 3, "rand2": 5, "best2": 4, "currenttobest1": 2, "randtobest1": 3}


def _mut(name, F, best, xi, x):
    f = np.float32
    F = f(F)
    d = lambda a, b: f(a - b)  # noqa: E731
    if name == "best1":
        return f(best) + F * d(x[0], x[1])
    if name == "rand1":
        return f(x[0]) + F * d(x[1], x[2])
    if name == "rand2":
        return (f(x[0]) + F * d(x[1], x[2])) + F * d(x[3], x[4])
    if name == "best2":
        return (f(best) + F * d(x[0], x[1])) + F * d(x[2], x[3])
    if name == "currenttobest1":
        return (f(xi) + F * d(best, xi)) + F * d(x[0], x[1])
    return (f(x[0]) + F * d(best, x[0])) + F * d(x[1], x[2])


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    sd = W.tiny_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    return sd, sp, keys, W.lognormal_table(len(keys), seed=0)


@pytest.mark.parametrize("mutation", list(PARTNERS))
@pytest.mark.parametrize("F", [1.0, 0.7])
def test_de_mutation_is_the_formula_for_some_ordering_of_the_partners(oracle_mod, tiny, mutation, F):
    sd, sp, keys, table = tiny
    O = oracle_mod
    r = np.array(sd.n_values)
    P = PARTNERS[mutation] + 1
    checked = 0
    for seed in range(6):
        T = O.run("de", sp, keys, table, pop=P, gens=2, seed=seed, de_mutation=mutation, de_F=F, de_CR=1.0)
        for g in (1, 2):
            X = O.unpack(sp, T["popk"][g - 1])
            best = O.unpack(sp, T["best_key"][g - 1:g])[0]
            for i in range(P):
                others = [X[j] for j in range(P) if j != i]
                got = T["cand"][g][i]
                ok = False
                for perm in itertools.permutations(others):
                    m = _mut(mutation, F, best, X[i], perm)
                    v = np.clip(np.rint(m), 0, r - 1).astype(np.int64)
                    if O.pack(sp, v[None, :])[0] == got:
                        ok = True
                        break
                assert ok, (mutation, seed, g, i)
                checked += 1
    assert checked == 12 * P


@pytest.mark.parametrize("mutation", ["rand1", "best2"])
def test_crossover_extremes(oracle_mod, tiny, mutation):
    sd, sp, keys, table = tiny
    O = oracle_mod
    # CR = 1: both crossovers take every gene from the mutant, so the runs coincide
    a = O.run("de", sp, keys, table, pop=12, gens=20, seed=3, de_mutation=mutation, de_CR=1.0)
    b = O.run("de", sp, keys, table, pop=12, gens=20, seed=3, de_mutation=mutation, de_CR=1.0, de_crossover="exp")
    for f in ("cand", "evalk", "popk", "best_key"):
        assert np.array_equal(a[f], b[f]), f
    # CR = 0: one gene from the mutant, the others from the target
    for cx in ("bin", "exp"):
        T = O.run("de", sp, keys, table, pop=12, gens=6, seed=4, de_mutation=mutation, de_CR=0.0, de_crossover=cx)
        for g in (1, 2):
            d = (O.unpack(sp, T["cand"][g]) != O.unpack(sp, T["popk"][g - 1])).sum(axis=1)
            assert (d <= 1).all(), cx


def test_exponential_crossover_copies_one_cyclic_window(oracle_mod):
    """With F = 0 the rand1 mutant is partner x0 itself, so an exponential-crossover trial must be
    the target with one cyclic window of genes taken from some other member, and the window
    (the start gene plus every further gene while the draws stay below CR) averages about
    1 + CR / (1 - CR) genes."""
    sd = W._space("free8", [(f"p{k}", list(range(5))) for k in range(8)], [])
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    table = W.lognormal_table(len(keys), seed=2)
    L = np.arange(1, 9)
    win = np.zeros((8, 8, 8), bool)                      # [start, length - 1, gene]
    for s0 in range(8):
        for li, ln in enumerate(L):
            win[s0, li, (s0 + np.arange(ln)) % 8] = True
    windows = []
    for seed in range(60):
        T = oracle_mod.run("de", sp, keys, table, pop=4, gens=1, seed=seed, de_mutation="rand1", de_F=0.0,
                           de_CR=0.5, de_crossover="exp")
        t = oracle_mod.unpack(sp, T["cand"][1])
        x = oracle_mod.unpack(sp, T["popk"][0])
        for i in range(4):
            fits = [L[li] for j in range(4) if j != i
                    for s0, li in zip(*np.nonzero((np.where(win, x[j], x[i]) == t[i]).all(axis=2)))]
            assert fits, (seed, i)
            windows.append(min(fits))
    assert 1.6 < np.mean(windows) < 2.4
    assert max(windows) >= 4


def _pairs_ok(kind, c0, c1, X):
    N = len(c0)
    for A in X:
        for B in X:
            m = c0 != A
            if not ((c0 == A) | (c0 == B)).all() or not (np.where(c0 == A, c1 == B, c1 == A)).all():
                continue
            if kind == "single_point":
                if any((c0 == np.r_[A[:k], B[k:]]).all() and (c1 == np.r_[B[:k], A[k:]]).all() for k in range(1, N)):
                    return True
            elif kind == "two_point":
                for lo in range(1, N - 1):
                    for hi in range(lo + 1, N):
                        if (c0 == np.r_[A[:lo], B[lo:hi], A[hi:]]).all() and (c1 == np.r_[B[:lo], A[lo:hi], B[hi:]]).all():
                            return True
            elif kind == "uniform":
                return True
            else:
                D = int((A != B).sum())
                if int(m.sum()) == D // 2:
                    return True
    return False


@pytest.mark.parametrize("kind", ["single_point", "two_point", "uniform", "disruptive_uniform"])
def test_ga_children_come_from_two_members_by_the_variant(oracle_mod, kind):
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    table = W.smooth_table(sd, oracle_mod.unpack(sp, keys), seed=0)
    swapped = []
    for seed in range(3):
        T = oracle_mod.run("ga", sp, keys, table, pop=20, gens=2, seed=seed, ga_crossover=kind)
        for g in (1, 2):
            X = oracle_mod.unpack(sp, T["popk"][g - 1])
            C = oracle_mod.unpack(sp, T["cand"][g])
            for c in range(10):
                assert _pairs_ok(kind, C[2 * c], C[2 * c + 1], X), (kind, seed, g, c)
                swapped.append(int((C[2 * c] != C[2 * c + 1]).sum()))
    assert max(swapped) > 0
