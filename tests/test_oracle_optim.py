"""Pins of the oracle's four constraint-aware optimizers.

The paper prints no optimizer trace, so trajectories are pinned only by reduction cases
(Section IV-B..IV-D read at degenerate hyper-parameters), invariants and rerun determinism.
"""
import numpy as np
import pytest

from paper_2606_28372_b300 import workloads as W

MUT_PICK, CROSS, GA_SEL, GA_CUT = 2, 3, 6, 7


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    sd = W.tiny_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    return sd, sp, keys, W.lognormal_table(len(keys), seed=0)


@pytest.fixture(scope="module")
def medium(oracle_mod):
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    return sd, sp, keys, W.smooth_table(sd, oracle_mod.unpack(sp, keys), seed=0)


def _common_invariants(O, sp, keys, table, T):
    evk = T["evalk"]
    G1, P = evk.shape
    rk = O.lookup(keys, evk.ravel()).reshape(evk.shape)
    assert (rk >= 0).all()                                   # only valid configs are evaluated
    assert np.array_equal(T["fit"], table[rk])               # fitness is the table entry
    for g in range(G1):                                      # memoised unique count
        assert T["n_unique"][g] == len(np.unique(evk[: g + 1]))
        f = T["fit"][: g + 1].ravel()
        k = evk[: g + 1].ravel()
        m = f.min()
        assert T["best_fit"][g] == m and T["best_key"][g] == k[f == m].min()


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
def test_invariants_and_determinism(oracle_mod, tiny, kind):
    sd, sp, keys, table = tiny
    T = oracle_mod.run(kind, sp, keys, table, pop=20, gens=100, seed=0)
    _common_invariants(oracle_mod, sp, keys, table, T)
    T2 = oracle_mod.run(kind, sp, keys, table, pop=20, gens=100, seed=0)
    for f in T:
        assert np.array_equal(T[f], T2[f]), f
    T3 = oracle_mod.run(kind, sp, keys, table, pop=20, gens=100, seed=1)
    assert not np.array_equal(T["cand"], T3["cand"])
    # the initial population is one valid rank per stratum
    nv, P = len(keys), 20
    rk = oracle_mod.lookup(keys, T["cand"][0])
    lo = (np.arange(P) * nv) // P
    hi = (np.arange(1, P + 1) * nv) // P
    assert ((rk >= lo) & (rk < hi)).all()


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
def test_invariants_medium(oracle_mod, medium, kind):
    sd, sp, keys, table = medium
    T = oracle_mod.run(kind, sp, keys, table, pop=32, gens=6, seed=3)
    _common_invariants(oracle_mod, sp, keys, table, T)


def test_de_population_rules(oracle_mod, tiny):
    """Greedy selection never worsens a member, members stay distinct, and two generations
    without any acceptance trigger a re-draw of the population (Section IV-B)."""
    sd, sp, keys, table = tiny
    T = oracle_mod.run("de", sp, keys, table, pop=20, gens=100, seed=4)
    stag, pending, reinits = 0, False, 0
    for g in range(1, 101):
        assert len(np.unique(T["popk"][g])) == 20
        if pending:
            assert np.array_equal(T["popk"][g], T["evalk"][g])
            assert np.array_equal(T["cand"][g], T["rep"][g])
            pending, stag, reinits = False, 0, reinits + 1
            continue
        assert (T["popf"][g] <= T["popf"][g - 1]).all()
        acc = int(np.sum(T["popk"][g] != T["popk"][g - 1]))
        stag = 0 if acc else stag + 1
        if stag >= 2:
            pending, stag = True, 0
    assert reinits >= 0


def test_de_f0_cr0_single_gene_from_best(oracle_mod, tiny):
    """F=0 makes the mutant equal to best; CR=0 takes exactly gene j_rand from it."""
    sd, sp, keys, table = tiny
    seed = 9
    T = oracle_mod.run("de", sp, keys, table, pop=20, gens=1, seed=seed, de_F=0.0, de_CR=0.0)
    f0, k0 = T["popf"][0], T["popk"][0]
    best = k0[np.flatnonzero(f0 == f0.min())[-1]]     # Algorithm 1 updates best on f <= f(best)
    ib = oracle_mod.unpack(sp, [best])[0]
    for i in range(20):
        x = oracle_mod.unpack(sp, [k0[i]])[0]
        u = oracle_mod.unpack(sp, [T["cand"][1][i]])[0]
        jr = (oracle_mod.rng_word(seed, i, 1, CROSS, 0) * sp.n) >> 32
        want = x.copy()
        want[jr] = ib[jr]
        assert np.array_equal(u, want)


def test_de_f0_cr1_stagnation_reinit(oracle_mod, tiny):
    """F=0, CR=1: every trial equals best, which is already in X, so nothing is accepted; after
    two such generations the population is re-drawn."""
    sd, sp, keys, table = tiny
    T = oracle_mod.run("de", sp, keys, table, pop=20, gens=4, seed=2, de_F=0.0, de_CR=1.0)
    f0, k0 = T["popf"][0], T["popk"][0]
    best = k0[np.flatnonzero(f0 == f0.min())[-1]]
    assert (T["cand"][1] == best).all() and (T["cand"][2] == best).all()
    assert np.array_equal(T["popk"][2], k0)
    assert np.array_equal(T["popk"][3], T["evalk"][3]) and not np.array_equal(T["popk"][3], k0)
    nv = len(keys)
    rk = oracle_mod.lookup(keys, T["cand"][3])
    lo = (np.arange(20) * nv) // 20
    assert ((rk >= lo) & (rk < (np.arange(1, 21) * nv) // 20)).all()


def test_pso_zero_coefficients_stationary(oracle_mod, medium):
    sd, sp, keys, table = medium
    T = oracle_mod.run("pso", sp, keys, table, pop=16, gens=5, seed=1, pso_w=0.0, pso_c1=0.0, pso_c2=0.0)
    for g in range(1, 6):
        assert np.array_equal(T["pos"][g], T["pos"][0])
        assert np.array_equal(T["cand"][g], T["cand"][0])   # snap of a grid point is itself


def test_pso_pbest_monotone(oracle_mod, medium):
    sd, sp, keys, table = medium
    T = oracle_mod.run("pso", sp, keys, table, pop=32, gens=8, seed=5)
    assert (np.diff(T["popf"], axis=0) <= 0).all()


def test_firefly_equal_brightness_no_attraction(oracle_mod, medium):
    sd, sp, keys, table = medium
    flat = np.ones(len(keys), np.float32)
    T = oracle_mod.run("firefly", sp, keys, flat, pop=16, gens=4, seed=1)
    for g in range(1, 5):
        assert np.array_equal(T["pos"][g], T["pos"][0])


def test_ga_no_mutation_full_space_is_plain_crossover(oracle_mod):
    """Without constraints every child is valid; with p_mut = 0 the children are exactly the
    single-point crossovers of the beta-selected parents of the (fitness, key)-sorted population."""
    vals = [[1, 2, 3, 4], [1, 2], [5, 6, 7], [0, 1, 2, 3, 4]]
    sp = oracle_mod.make_space(["a", "b", "c", "d"], vals, [])
    keys = oracle_mod.valid_keys(sp)
    table = W.lognormal_table(len(keys), seed=3)
    P, seed = 10, 21
    T = oracle_mod.run("ga", sp, keys, table, pop=P, gens=3, seed=seed, ga_pmut=0.0)
    for g in range(1, 4):
        X, F = T["popk"][g - 1], T["popf"][g - 1]
        order = sorted(range(P), key=lambda i: (float(F[i]), int(X[i])))
        for c in range(P // 2):
            a = order[oracle_mod.beta_pick(oracle_mod.rng_word(seed, c, g, GA_SEL, 0), P)]
            b = order[oracle_mod.beta_pick(oracle_mod.rng_word(seed, c, g, GA_SEL, 1), P)]
            cut = 1 + ((oracle_mod.rng_word(seed, c, g, GA_CUT, 0) * (sp.n - 1)) >> 32)
            A, B = oracle_mod.unpack(sp, [X[a], X[b]])
            c0 = np.concatenate([A[:cut], B[cut:]])
            c1 = np.concatenate([B[:cut], A[cut:]])
            got = oracle_mod.unpack(sp, T["cand"][g][2 * c: 2 * c + 2])
            assert np.array_equal(got[0], c0) and np.array_equal(got[1], c1)
        assert np.array_equal(T["cand"][g], T["evalk"][g])


def test_ga_mutation_is_a_valid_hamming_neighbour(oracle_mod, tiny):
    sd, sp, keys, table = tiny
    T = oracle_mod.run("ga", sp, keys, table, pop=20, gens=30, seed=8, ga_pmut=1.0)
    kset = set(int(k) for k in keys)
    moved = 0
    for g in range(1, 31):
        for a, b in zip(T["rep"][g], T["evalk"][g]):
            d = int(np.sum(oracle_mod.unpack(sp, [a])[0] != oracle_mod.unpack(sp, [b])[0]))
            assert d == 1 and int(b) in kset
            moved += 1
    assert moved == 600


def test_target_hit_recorded(oracle_mod, tiny):
    sd, sp, keys, table = tiny
    opt = float(table.min())
    T = oracle_mod.run("de", sp, keys, table, pop=20, gens=100, seed=0, target=np.float32(1.01 * opt))
    g = int(T["hit"][0])
    if g >= 0:
        assert T["best_fit"][g] <= np.float32(1.01 * opt)
        assert g == 0 or T["best_fit"][g - 1] > np.float32(1.01 * opt)
        assert T["hit"][1] == T["n_unique"][g]
