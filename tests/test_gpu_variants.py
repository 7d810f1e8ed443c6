"""GPU parity of the DE and GA operator variants (Sections IV-B, IV-D): whole trajectories step by
step and in batches, bit-exact against the oracle."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64
from tests.test_gpu_rules import step_trace

pytestmark = pytest.mark.gpu

DE_MUT = ["best1", "rand1", "rand2", "best2", "currenttobest1", "randtobest1"]
GA_CX = ["single_point", "two_point", "uniform", "disruptive_uniform"]
FIELDS = ("cand", "evalk", "fit", "popk", "popf", "best_key", "best_fit", "n_unique")


@pytest.fixture(scope="module")
def spaces(oracle_mod):
    return {n: Pair(sd, oracle_mod) for n, sd in (("tiny", W.tiny_space()), ("medium", W.medium_space()))}


def _same(T, E):
    for f in FIELDS:
        a, b = T[f], E[f].astype(T[f].dtype)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{f} differs first at {bad[0]} ({len(bad)} entries)")


@pytest.mark.parametrize("mutation", DE_MUT)
@pytest.mark.parametrize("crossover", ["bin", "exp"])
@pytest.mark.parametrize("name,pop,gens", [("tiny", 8, 30), ("medium", 48, 12)])
def test_de_variant_trajectory(oracle_mod, spaces, mutation, crossover, name, pop, gens):
    p = spaces[name]
    kw = dict(de_mutation=mutation, de_crossover=crossover)
    E = oracle_mod.run("de", p.osp, p.okeys, p.table, pop=pop, gens=gens, seed=21, **kw)
    T = step_trace(p, "de", pop, gens, 21, **kw)
    _same(T, E)


@pytest.mark.parametrize("crossover", GA_CX)
@pytest.mark.parametrize("name,pop,gens", [("tiny", 20, 25), ("medium", 48, 12)])
@pytest.mark.parametrize("aware", [1, 0])
def test_ga_variant_trajectory(oracle_mod, spaces, crossover, name, pop, gens, aware):
    p = spaces[name]
    kw = dict(ga_crossover=crossover, constraint_aware=aware)
    E = oracle_mod.run("ga", p.osp, p.okeys, p.table, pop=pop, gens=gens, seed=22, **kw)
    T = step_trace(p, "ga", pop, gens, 22, **kw)
    _same(T, E)


def test_variants_in_a_batch(oracle_mod, spaces):
    from paper_2606_28372_b300 import catune as ct
    pairs = [spaces["medium"], spaces["tiny"]]
    runs = [(0, "de", 64, 5, -np.inf), (1, "de", 16, 6, -np.inf), (0, "ga", 40, 7, -np.inf), (1, "ga", 20, 8, -np.inf)]
    kw = dict(de_mutation="randtobest1", de_crossover="exp", ga_crossover="disruptive_uniform")
    b = ct.Batch([q.sp for q in pairs], runs, **kw)
    gens = 10
    for _ in range(gens):
        b.step()
    for r, (si, kind, pop, seed, _) in enumerate(runs):
        q = pairs[si]
        E = oracle_mod.run(kind, q.osp, q.okeys, q.table, pop=pop, gens=gens - 1, seed=seed, **kw)
        k = torch.empty(pop, dtype=torch.int64, device="cuda")
        f = torch.empty(pop, dtype=torch.float32, device="cuda")
        b.run_state(r, k, f)
        assert np.array_equal(from_dev_u64(k), E["popk"][-1]), kind
        assert np.array_equal(f.cpu().numpy(), E["popf"][-1]), kind


def test_too_small_population_is_refused(spaces):
    from paper_2606_28372_b300 import catune as ct
    with pytest.raises(ct.CatuneError):
        ct.Opt(spaces["tiny"].sp, "de", 5, 1, de_mutation="rand2")
    ct.Opt(spaces["tiny"].sp, "de", 6, 1, de_mutation="rand2")
    with pytest.raises(ct.CatuneError):
        ct.Batch([spaces["tiny"].sp], [(0, "de", 4, 1, -np.inf)], de_mutation="best2")
