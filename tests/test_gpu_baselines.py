"""GPU parity of the non-constraint-aware baselines (random Cartesian start, no repair, static
penalty, plain GA mutation): single runs step by step and as a graph, and batched runs."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64
from tests.test_gpu_rules import step_trace

pytestmark = pytest.mark.gpu

FIELDS = ("cand", "evalk", "fit", "popk", "popf", "best_key", "best_fit", "n_unique")


@pytest.fixture(scope="module")
def spaces(oracle_mod):
    free = W._space("free", [(p, v) for p, v in W.tiny_space().params], [])
    return {n: Pair(sd, oracle_mod) for n, sd in (("tiny", W.tiny_space()), ("medium", W.medium_space()),
                                                   ("b9", W.batched_space(9)), ("free", free))}


def _same(T, E, kind):
    for f in FIELDS + (("pos",) if kind in ("pso", "firefly") else ()):
        a, b = T[f], E[f].astype(T[f].dtype)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{f} differs first at {bad[0]} ({len(bad)} entries)")


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
@pytest.mark.parametrize("name,pop,gens", [("tiny", 20, 30), ("medium", 64, 12), ("b9", 32, 12), ("free", 16, 10)])
def test_unaware_trajectory_matches_oracle(oracle_mod, spaces, kind, name, pop, gens):
    p = spaces[name]
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=pop, gens=gens, seed=11, constraint_aware=0)
    T = step_trace(p, kind, pop, gens, 11, constraint_aware=0)
    _same(T, E, kind)
    if name == "medium":
        assert (T["fit"] == np.float32(1e20)).any()     # the dense-constraint space penalises


@pytest.mark.parametrize("kind", ["de", "ga"])
def test_unaware_graph_equals_steps(spaces, kind):
    from paper_2606_28372_b300 import catune as ct
    p = spaces["medium"]
    a = ct.Opt(p.sp, kind, 64, 3, constraint_aware=0)
    b = ct.Opt(p.sp, kind, 64, 3, constraint_aware=0)
    for g in range(16):
        a.step(g)
    b.run_graph(0, 16)
    ka, kb = (torch.empty(64, dtype=torch.int64, device="cuda") for _ in range(2))
    fa, fb = (torch.empty(64, dtype=torch.float32, device="cuda") for _ in range(2))
    a.state(ka, fa)
    b.state(kb, fb)
    assert np.array_equal(from_dev_u64(ka), from_dev_u64(kb)) and torch.equal(fa, fb)
    assert a.best() == b.best()


def test_unaware_batch_matches_oracle(oracle_mod, spaces):
    from paper_2606_28372_b300 import catune as ct
    pairs = [spaces["b9"], spaces["medium"], spaces["tiny"]]
    runs = [(0, "de", 64, 7, -np.inf), (1, "ga", 96, 8, -np.inf), (2, "pso", 32, 9, -np.inf),
            (0, "firefly", 32, 10, -np.inf), (1, "de", 32, 12, -np.inf)]
    b = ct.Batch([q.sp for q in pairs], runs, constraint_aware=0)
    gens = 10
    for _ in range(gens):
        b.step()
    res = b.results()
    for r, (si, kind, pop, seed, _) in enumerate(runs):
        q = pairs[si]
        E = oracle_mod.run(kind, q.osp, q.okeys, q.table, pop=pop, gens=gens - 1, seed=seed, constraint_aware=0)
        k = torch.empty(pop, dtype=torch.int64, device="cuda")
        f = torch.empty(pop, dtype=torch.float32, device="cuda")
        b.run_state(r, k, f)
        assert np.array_equal(from_dev_u64(k), E["popk"][-1]), kind
        assert np.array_equal(f.cpu().numpy(), E["popf"][-1]), kind
        assert int(res["n_unique"][r]) == int(E["n_unique"][-1]), kind
        assert int(res["best_key"][r]) == int(E["best_key"][-1]), kind


def test_surrogate_needs_the_constraint_aware_method(spaces):
    from paper_2606_28372_b300 import catune as ct
    o = ct.Opt(spaces["tiny"].sp, "de", 32, 1, constraint_aware=0)
    with pytest.raises(ct.CatuneError):
        o.set_surrogate(torch.log(spaces["tiny"].dtable))
