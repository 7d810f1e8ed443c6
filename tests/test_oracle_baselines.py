"""Pins of the oracle's non-constraint-aware baselines (Sections IV-B/IV-C, the comparison of
Section V): random start over the Cartesian product, no repair, a static penalty for invalid
configurations, and a GA mutation that ignores the constraints.

The pins are statistical facts of uniform sampling (marginals, the valid fraction equals the
density of the space), the penalty semantics (invalid configurations cost the penalty and are
never counted as evaluated), and the shape of one mutation (exactly one parameter changes).
"""
import numpy as np
import pytest
from scipy import stats

from paper_2606_28372_b300 import workloads as W

PENALTY = np.float32(1e20)


@pytest.fixture(scope="module")
def medium(oracle_mod):
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    return sd, sp, keys, W.smooth_table(sd, oracle_mod.unpack(sp, keys), seed=0)


@pytest.mark.parametrize("kind", ["de", "ga"])
def test_start_is_uniform_over_the_cartesian_product(oracle_mod, medium, kind):
    sd, sp, keys, table = medium
    P = 1024
    T = oracle_mod.run(kind, sp, keys, table, pop=P, gens=0, seed=5, constraint_aware=0)
    tup = oracle_mod.unpack(sp, T["cand"][0])
    r = np.array(sd.n_values)
    assert ((tup >= 0) & (tup < r)).all()
    for k in range(len(r)):                                    # each marginal is uniform
        cnt = np.bincount(tup[:, k], minlength=r[k])
        assert stats.chisquare(cnt).pvalue > 1e-4, (k, cnt)
    rho = len(keys) / sd.cartesian_size                        # valid fraction = density
    n_valid = int((oracle_mod.lookup(keys, T["cand"][0]) >= 0).sum())
    sd_ = np.sqrt(P * rho * (1 - rho))
    assert abs(n_valid - P * rho) < 5 * sd_ + 1
    # constraint-aware start: every member valid
    Ta = oracle_mod.run(kind, sp, keys, table, pop=P, gens=0, seed=5)
    assert (oracle_mod.lookup(keys, Ta["cand"][0]) >= 0).all()


@pytest.mark.parametrize("kind", ["pso", "firefly"])
def test_swarm_start_is_uniform_in_the_unit_cube(oracle_mod, medium, kind):
    sd, sp, keys, table = medium
    T = oracle_mod.run(kind, sp, keys, table, pop=512, gens=0, seed=6, constraint_aware=0)
    x = T["pos"][0]
    assert ((x >= 0) & (x < 1)).all()
    assert stats.kstest(x.ravel().astype(np.float64), "uniform").pvalue > 1e-4


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
def test_no_repair_and_static_penalty(oracle_mod, medium, kind):
    sd, sp, keys, table = medium
    T = oracle_mod.run(kind, sp, keys, table, pop=32, gens=25, seed=1, constraint_aware=0)
    assert np.array_equal(T["rep"], T["cand"])                 # candidates are evaluated as proposed
    if kind != "ga":
        assert np.array_equal(T["evalk"], T["rep"])
    evk = T["evalk"]
    rk = oracle_mod.lookup(keys, evk.ravel()).reshape(evk.shape)
    bad = rk < 0
    assert bad.any()
    assert (T["fit"][bad] == PENALTY).all()
    assert np.array_equal(T["fit"][~bad], table[rk[~bad]])
    for g in range(evk.shape[0]):                              # only valid configurations count
        assert T["n_unique"][g] == len(np.unique(evk[: g + 1][~bad[: g + 1]]))
        f = T["fit"][: g + 1].ravel()
        m = f.min()
        assert T["best_fit"][g] == m and T["best_key"][g] == evk[: g + 1].ravel()[f == m].min()


def test_de_selection_never_trades_a_valid_member_for_a_penalised_one(oracle_mod, medium):
    sd, sp, keys, table = medium
    T = oracle_mod.run("de", sp, keys, table, pop=32, gens=40, seed=2, constraint_aware=0)
    checked = 0
    for g in range(1, 41):
        if np.array_equal(T["popk"][g], T["evalk"][g]):        # a stagnation restart replaces all
            continue
        prev, cur = T["popf"][g - 1], T["popf"][g]
        assert (cur <= prev).all()
        assert not ((prev < PENALTY) & (cur == PENALTY)).any()
        checked += 1
    assert checked > 20


@pytest.mark.parametrize("pmut", [0.0, 1.0])
def test_plain_ga_mutation_changes_exactly_one_parameter(oracle_mod, medium, pmut):
    sd, sp, keys, table = medium
    T = oracle_mod.run("ga", sp, keys, table, pop=32, gens=20, seed=3, ga_pmut=pmut, constraint_aware=0)
    a = oracle_mod.unpack(sp, T["rep"][1:].ravel())
    b = oracle_mod.unpack(sp, T["evalk"][1:].ravel())
    nd = (a != b).sum(axis=1)
    if pmut == 0.0:
        assert (nd == 0).all()
    else:
        assert (nd == 1).all()
        assert ((b >= 0) & (b < np.array(sd.n_values))).all()


def test_plain_ga_mutation_rate(oracle_mod, medium):
    sd, sp, keys, table = medium
    T = oracle_mod.run("ga", sp, keys, table, pop=64, gens=40, seed=4, constraint_aware=0)
    n = T["rep"][1:].size
    m = int((T["rep"][1:] != T["evalk"][1:]).sum())
    assert abs(m - 0.2 * n) < 5 * np.sqrt(n * 0.2 * 0.8)


def test_unconstrained_space_sees_no_penalty(oracle_mod):
    sd = W._space("free", [(p, v) for p, v in W.tiny_space().params], [])
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    assert len(keys) == sd.cartesian_size
    table = W.lognormal_table(len(keys), seed=1)
    for kind in ["de", "pso", "firefly", "ga"]:
        T = oracle_mod.run(kind, sp, keys, table, pop=16, gens=15, seed=0, constraint_aware=0)
        assert (oracle_mod.lookup(keys, T["evalk"].ravel()) >= 0).all()
        assert (T["fit"] < PENALTY).all()
