"""GPU parity of the batched form: each run of the persistent launches (one generation per
launch, or many generations of each run per launch) equals the same run done alone (and the
oracle), for every optimizer, population and space size."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64

pytestmark = pytest.mark.gpu

KINDS = ["de", "pso", "ga", "firefly"]


@pytest.fixture(scope="module")
def spaces(oracle_mod):
    return [Pair(W.batched_space(s), oracle_mod, table="smooth", seed=s) for s in (0, 9, 17, 31)]


def _runs(pairs, n):
    runs = []
    for r in range(n):
        si = r % len(pairs)
        tgt = float(np.float32(1.01 * float(pairs[si].table.min())))
        runs.append((si, KINDS[r % 4], 32 * (1 + (r // 4) % 4), 1000 + r, tgt))
    return runs


def _single(pair, kind, pop, seed, target, gens):
    from paper_2606_28372_b300 import catune as ct
    o = ct.Opt(pair.sp, kind, pop, seed, target=target)
    for g in range(gens):
        o.step(g)
    k = torch.empty(pop, dtype=torch.int64, device="cuda")
    f = torch.empty(pop, dtype=torch.float32, device="cuda")
    o.state(k, f)
    return from_dev_u64(k), f.cpu().numpy(), o.best()


@pytest.mark.parametrize("mode", ["step", "graph", "mixed", "graph_per_generation"])
def test_batch_equals_single_runs(spaces, mode):
    from paper_2606_28372_b300 import catune as ct
    runs = _runs(spaces, 24)
    b = ct.Batch([p.sp for p in spaces], runs)
    gens = 12
    if mode == "step":
        for _ in range(gens):
            b.step()
    elif mode == "graph":
        b.run_graph(1)
        b.run_graph(gens - 1)
    elif mode == "graph_per_generation":   # one persistent launch per generation, captured
        b.set_gens_per_launch(1)
        b.run_graph(5)
        b.set_gens_per_launch(3)
        b.run_graph(gens - 5)
    else:   # launches of 1, 4 and 3 generations in turn
        for _ in range(3):
            b.step()
        b.run_graph(4)
        b.step()
        b.run_graph(4)
    res = b.results()
    for r, (si, kind, pop, seed, tgt) in enumerate(runs):
        k = torch.empty(pop, dtype=torch.int64, device="cuda")
        f = torch.empty(pop, dtype=torch.float32, device="cuda")
        b.run_state(r, k, f)
        sk, sf, sb = _single(spaces[si], kind, pop, seed, tgt, gens)
        assert np.array_equal(from_dev_u64(k), sk), (r, kind)
        assert np.array_equal(f.cpu().numpy(), sf), (r, kind)
        assert int(res["best_key"][r]) == sb["best_key"] and int(res["n_unique"][r]) == sb["n_unique"], (r, kind)
        assert int(res["hit_gen"][r]) == sb["hit_gen"] and int(res["hit_evals"][r]) == sb["hit_evals"], (r, kind)


def test_batch_equals_oracle(oracle_mod, spaces):
    from paper_2606_28372_b300 import catune as ct
    runs = [(1, "de", 64, 7, -np.inf), (3, "ga", 96, 8, -np.inf), (2, "pso", 32, 9, -np.inf), (0, "firefly", 32, 10, -np.inf)]
    b = ct.Batch([p.sp for p in spaces], runs)
    gens = 10
    for _ in range(gens):
        b.step()
    res = b.results()
    for r, (si, kind, pop, seed, _) in enumerate(runs):
        p = spaces[si]
        E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=pop, gens=gens - 1, seed=seed)
        k = torch.empty(pop, dtype=torch.int64, device="cuda")
        f = torch.empty(pop, dtype=torch.float32, device="cuda")
        b.run_state(r, k, f)
        assert np.array_equal(from_dev_u64(k), E["popk"][-1]), kind
        assert np.array_equal(f.cpu().numpy(), E["popf"][-1]), kind
        assert int(res["n_unique"][r]) == int(E["n_unique"][-1]) and int(res["best_key"][r]) == int(E["best_key"][-1])


def test_batch_launch_shapes_and_autotune(spaces, tmp_path):
    from paper_2606_28372_b300 import catune as ct
    runs = _runs(spaces, 40)
    b = ct.Batch([p.sp for p in spaces], runs)
    outs = []
    for th, cps in ((64, 2), (128, 3), (256, 1)):
        b.reset()
        b.set_launch(th, cps)
        for _ in range(6):
            b.step()
        outs.append(b.results())
    for o in outs[1:]:
        assert np.array_equal(o["best_key"], outs[0]["best_key"]) and np.array_equal(o["n_unique"], outs[0]["n_unique"])
    cache = str(tmp_path / "tune.jsonl")
    th, cps, ms = b.autotune(cache, gens=3)
    assert th in (64, 128, 256) and cps > 0 and ms > 0
    assert b.results()["n_unique"].sum() == 0            # left reset
    assert b.autotune(cache, gens=3)[:2] == (th, cps)    # cache hit
    for _ in range(6):
        b.step()
    assert np.array_equal(b.results()["best_key"], outs[0]["best_key"])


@pytest.mark.parametrize("mode,radius", [(1, 0), (2, 1)])
def test_batch_scan_paths_equal_oracle(oracle_mod, spaces, mode, radius):
    """Scan-only repair and a radius-1 ball: most pending candidates reach the in-CTA exhaustive
    scan (distance tables, chunks of 32, 16 and 8 candidates), against the oracle."""
    from paper_2606_28372_b300 import catune as ct
    runs = [(1, "de", 128, 17, -np.inf), (3, "ga", 96, 18, -np.inf), (2, "pso", 40, 19, -np.inf),
            (0, "de", 9, 20, -np.inf)]
    for p in spaces:
        p.sp.set_repair_mode(mode, radius)
    try:
        b = ct.Batch([p.sp for p in spaces], runs)
        gens = 6
        for _ in range(gens):
            b.step()
        res = b.results()
    finally:
        for p in spaces:
            p.sp.set_repair_mode(0, 0)
    for r, (si, kind, pop, seed, _) in enumerate(runs):
        p = spaces[si]
        E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=pop, gens=gens - 1, seed=seed)
        k = torch.empty(pop, dtype=torch.int64, device="cuda")
        b.run_state(r, k)
        assert np.array_equal(from_dev_u64(k), E["popk"][-1]), (kind, mode)
        assert int(res["n_unique"][r]) == int(E["n_unique"][-1]), (kind, mode)
