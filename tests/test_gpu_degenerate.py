"""Degenerate and extreme inputs for the optimizers, against the oracle: a space with one valid
configuration, a space whose parameters all have a single value (keys of zero bits), the
population bounds (3, and 1,024 for a single run), odd GA populations, the paper's repair rules
with nothing to choose from, and batches at their population bounds."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64
from tests.test_gpu_rules import step_trace

pytestmark = pytest.mark.gpu

KINDS = ["de", "pso", "firefly", "ga"]
FIELDS = ("cand", "evalk", "fit", "popk", "popf", "best_key", "best_fit", "n_unique")


def _same(T, E):
    for f in FIELDS:
        a, b = T[f], E[f].astype(T[f].dtype)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{f} differs first at {bad[0]} ({len(bad)} entries)")


@pytest.fixture(scope="module")
def spaces(oracle_mod):
    one = W._space("one_valid", [("a", [1, 2, 3]), ("b", [3, 4]), ("c", [0, 1, 2, 3])], ["a == 2 and b == 4 and c == 1"])
    point = W._space("point", [("a", [5]), ("b", [7]), ("c", [9])], [])
    return {"one": Pair(one, oracle_mod, table="lognormal"), "point": Pair(point, oracle_mod, table="lognormal"),
            "tiny": Pair(W.tiny_space(), oracle_mod), "medium": Pair(W.medium_space(), oracle_mod)}


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("aware", [1, 0])
@pytest.mark.parametrize("name", ["one", "point"])
def test_single_configuration_spaces(oracle_mod, spaces, kind, aware, name):
    p = spaces[name]
    assert len(p.okeys) == 1
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=3, gens=6, seed=1, constraint_aware=aware)
    T = step_trace(p, kind, 3, 6, 1, constraint_aware=aware)
    _same(T, E)
    if aware:
        assert (T["evalk"] == p.okeys[0]).all() and (T["n_unique"] == 1).all()


@pytest.mark.parametrize("kind", KINDS)
def test_largest_single_run_population(oracle_mod, spaces, kind):
    p = spaces["tiny"]
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=1024, gens=3, seed=2)
    T = step_trace(p, kind, 1024, 3, 2)
    _same(T, E)


@pytest.mark.parametrize("pop", [3, 21, 127])
def test_odd_ga_populations(oracle_mod, spaces, pop):
    p = spaces["medium"]
    E = oracle_mod.run("ga", p.osp, p.okeys, p.table, pop=pop, gens=5, seed=3)
    T = step_trace(p, "ga", pop, 5, 3)
    _same(T, E)


@pytest.mark.parametrize("kind", KINDS)
def test_paper_rules_with_one_valid_configuration(oracle_mod, spaces, kind):
    p = spaces["one"]
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=4, gens=5, seed=4, repair_rule=1)
    T = step_trace(p, kind, 4, 5, 4, repair_rule=1)
    _same(T, E)


def test_batch_population_bounds(oracle_mod, spaces):
    from paper_2606_28372_b300 import catune as ct
    pairs = [spaces["tiny"], spaces["one"], spaces["medium"]]
    runs = [(0, "de", 3, 1, -np.inf), (2, "ga", 256, 2, -np.inf), (1, "pso", 3, 3, -np.inf), (2, "firefly", 256, 4, -np.inf),
            (0, "ga", 3, 5, -np.inf)]
    b = ct.Batch([q.sp for q in pairs], runs)
    gens = 6
    for _ in range(gens):
        b.step()
    for r, (si, kind, pop, seed, _) in enumerate(runs):
        q = pairs[si]
        E = oracle_mod.run(kind, q.osp, q.okeys, q.table, pop=pop, gens=gens - 1, seed=seed)
        k = torch.empty(pop, dtype=torch.int64, device="cuda")
        b.run_state(r, k)
        assert np.array_equal(from_dev_u64(k), E["popk"][-1]), (kind, pop)
    with pytest.raises(ct.CatuneError):
        ct.Batch([spaces["tiny"].sp], [(0, "de", 257, 1, -np.inf)])
    with pytest.raises(ct.CatuneError):
        ct.Opt(spaces["tiny"].sp, "ga", 1025, 1)
