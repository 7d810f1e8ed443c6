"""GPU parity of the simulated clock (ct_set_eval_cost, ct_opt_cost) and of the batched
per-generation trace, and the score computed from GPU traces against the oracle's."""
import numpy as np
import pytest
import torch

from oracle import score as OS
from paper_2606_28372_b300 import score as PS
from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair

pytestmark = pytest.mark.gpu

P_EVENTS = 512


@pytest.fixture(scope="module")
def spaces(oracle_mod):
    out = []
    for sd in (W.medium_space(), W.batched_space(9), W.tiny_space()):
        p = Pair(sd, oracle_mod)
        p.cost = W.eval_cost_table(p.table, seed=5)
        p.dcost = torch.from_numpy(p.cost.view(np.int32)).cuda()
        p.sp.set_eval_cost(p.dcost)
        out.append(p)
    return out


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
@pytest.mark.parametrize("aware", [1, 0])
def test_single_run_clock_matches_oracle(oracle_mod, spaces, kind, aware):
    from paper_2606_28372_b300 import catune as ct
    p = spaces[0]
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=32, gens=12, seed=3, cost=p.cost, constraint_aware=aware)
    o = ct.Opt(p.sp, kind, 32, 3, constraint_aware=aware)
    for g in range(13):
        o.step(g)
        assert o.cost() == int(E["cost"][g]), g
    assert o.best()["n_unique"] == int(E["n_unique"][-1])


@pytest.mark.parametrize("aware", [1, 0])
@pytest.mark.parametrize("mode", ["step", "graph"])
def test_batch_trace_matches_oracle(oracle_mod, spaces, aware, mode):
    from paper_2606_28372_b300 import catune as ct
    runs = [(0, "de", 64, 7, -np.inf), (1, "ga", 20, 8, -np.inf), (2, "pso", 30, 9, -np.inf),
            (0, "firefly", 20, 10, -np.inf), (1, "de", 160, 11, -np.inf)]
    b = ct.Batch([q.sp for q in spaces], runs, constraint_aware=aware)
    G = 14
    b.set_trace(G, events=P_EVENTS)
    if mode == "step":
        for _ in range(G):
            b.step()
    else:
        b.run_graph(G)
    tr = b.trace()
    ev = b.events()
    for r, (si, kind, pop, seed, _) in enumerate(runs):
        q = spaces[si]
        E = oracle_mod.run(kind, q.osp, q.okeys, q.table, pop=pop, gens=G - 1, seed=seed, cost=q.cost,
                           constraint_aware=aware)
        assert np.array_equal(tr["cost"][r], E["cost"]), (r, kind)
        assert np.array_equal(tr["best_fit"][r], E["best_fit"]), (r, kind)
        assert np.array_equal(tr["n_unique"][r], E["n_unique"]), (r, kind)
        for a, f in zip(ev[r], ("ev_gen", "ev_idx", "ev_clock", "ev_fit")):
            assert np.array_equal(a, E[f].astype(a.dtype)), (r, kind, f)


def test_score_from_gpu_events_matches_oracle(oracle_mod, spaces):
    from paper_2606_28372_b300 import catune as ct
    q = spaces[1]
    G = 60
    runs = [(0, k, P, s, -np.inf) for s in range(4) for k, P in (("ga", 20), ("de", 160), ("pso", 30))]
    b = ct.Batch([q.sp], runs)
    b.set_trace(G, events=P_EVENTS)
    b.run_graph(G)
    ev = b.events()
    base = PS.Baseline(q.table, q.cost, 1000.0)
    for kind, P in (("ga", 20), ("de", 160), ("pso", 30)):
        rows = [r for r, run in enumerate(runs) if run[1] == kind]
        got = PS.run_scores(base, [ev[r] for r in rows], pop=P, overhead_us=1000.0)
        oev = []
        for r in rows:
            E = oracle_mod.run(kind, q.osp, q.okeys, q.table, pop=P, gens=G - 1, seed=runs[r][3], cost=q.cost)
            oev.append((E["ev_gen"], E["ev_idx"], E["ev_clock"], E["ev_fit"]))
        exp = OS.run_score(q.table, q.cost, oev, pop=P, overhead_us=1000.0)
        assert np.allclose(got["per_run"], exp["per_run"], rtol=1e-9, atol=1e-9), kind
        assert (got["per_run"] <= 1).all()
