"""GPU parity: optimizer trajectories (DE, PSO, Firefly, GA) equal the oracle's, generation by
generation and bit for bit: proposals, repaired keys, evaluated keys, fitness, population,
positions, best and unique-evaluation counts."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64

pytestmark = pytest.mark.gpu


def gpu_trace(p, kind, pop, gens, seed, **params):
    from paper_2606_28372_b300 import catune as ct
    opt = ct.Opt(p.sp, kind, pop, seed, **params)
    n = p.sd and len(p.sd.params)
    cand = torch.empty(pop, dtype=torch.int64, device="cuda")
    rep = torch.empty_like(cand)
    fit = torch.empty(pop, dtype=torch.float32, device="cuda")
    popk = torch.empty_like(cand)
    popf = torch.empty_like(fit)
    pos = torch.empty(pop * n, dtype=torch.float32, device="cuda")
    T = {k: [] for k in ("cand", "rep", "evalk", "fit", "popk", "popf", "pos", "best_key", "best_fit", "n_unique")}
    for g in range(gens + 1):
        opt.propose(g, cand)
        T["cand"].append(from_dev_u64(cand))
        p.sp.repair(cand, rep)
        T["rep"].append(from_dev_u64(rep))
        opt.post_repair(g, rep)
        T["evalk"].append(from_dev_u64(rep))
        p.sp.evaluate(rep, fit, opt=opt)
        T["fit"].append(fit.cpu().numpy())
        opt.select(g, rep, fit)
        opt.state(popk, popf, pos)
        T["popk"].append(from_dev_u64(popk))
        T["popf"].append(popf.cpu().numpy())
        T["pos"].append(pos.cpu().numpy().reshape(pop, n))
        b = opt.best()
        T["best_key"].append(b["best_key"])
        T["best_fit"].append(np.float32(b["best_fit"]))
        T["n_unique"].append(b["n_unique"])
    return {k: np.array(v) for k, v in T.items()}, opt


def compare(T, E, kind):
    fields = ["cand", "rep", "evalk", "fit", "popk", "popf", "best_key", "best_fit", "n_unique"]
    if kind in ("pso", "firefly"):
        fields.append("pos")
    for f in fields:
        a, b = T[f], E[f].astype(T[f].dtype) if f != "pos" else E[f]
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{f} differs first at {bad[0]} ({len(bad)} entries)")


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    return Pair(W.tiny_space(), oracle_mod)


@pytest.fixture(scope="module")
def medium(oracle_mod):
    return Pair(W.medium_space(), oracle_mod)


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
def test_tiny_trajectory(oracle_mod, tiny, kind):
    """Tiny space, pop 20, 100 generations (the DE configuration of the tiny workload)."""
    E = oracle_mod.run(kind, tiny.osp, tiny.okeys, tiny.table, pop=20, gens=100, seed=0)
    T, _ = gpu_trace(tiny, kind, 20, 100, 0)
    compare(T, E, kind)


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
@pytest.mark.parametrize("seed", [0, 1])
def test_medium_trajectory(oracle_mod, medium, kind, seed):
    """Medium space, pop 128 (the four-optimizer workload), first 12 generations."""
    E = oracle_mod.run(kind, medium.osp, medium.okeys, medium.table, pop=128, gens=12, seed=seed)
    T, _ = gpu_trace(medium, kind, 128, 12, seed)
    compare(T, E, kind)


@pytest.mark.parametrize("kind", ["de", "ga"])
def test_reduction_cases_match(oracle_mod, tiny, kind):
    prm = dict(de_F=0.0, de_CR=0.0) if kind == "de" else dict(ga_pmut=1.0)
    E = oracle_mod.run(kind, tiny.osp, tiny.okeys, tiny.table, pop=20, gens=20, seed=3, **prm)
    T, _ = gpu_trace(tiny, kind, 20, 20, 3, **prm)
    compare(T, E, kind)


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
def test_graph_and_step_equal_trace(oracle_mod, medium, kind):
    """Whole generations through ct_opt_step and through a replayed CUDA graph end in the same
    state as the oracle."""
    from paper_2606_28372_b300 import catune as ct
    gens = 10
    E = oracle_mod.run(kind, medium.osp, medium.okeys, medium.table, pop=64, gens=gens, seed=7)
    a = ct.Opt(medium.sp, kind, 64, 7)
    for g in range(gens + 1):
        a.step(g)
    b = ct.Opt(medium.sp, kind, 64, 7)
    b.run_graph(0, 1)
    for g in range(1, gens + 1, 5):
        b.run_graph(g, 5)
    for o in (a, b):
        k = torch.empty(64, dtype=torch.int64, device="cuda")
        f = torch.empty(64, dtype=torch.float32, device="cuda")
        o.state(k, f)
        assert np.array_equal(from_dev_u64(k), E["popk"][gens])
        assert np.array_equal(f.cpu().numpy(), E["popf"][gens])
        bb = o.best()
        assert bb["best_key"] == int(E["best_key"][gens]) and bb["n_unique"] == int(E["n_unique"][gens])


def test_checkpoint_resume(oracle_mod, medium):
    from paper_2606_28372_b300 import catune as ct
    a = ct.Opt(medium.sp, "de", 32, 11)
    for g in range(9):
        a.step(g)
    blob = a.save()
    b = ct.Opt(medium.sp, "de", 32, 11)
    b.load(blob)
    for g in range(9, 17):
        a.step(g)
        b.step(g)
    assert a.best() == b.best()
    ka, kb = (torch.empty(32, dtype=torch.int64, device="cuda") for _ in range(2))
    a.state(ka)
    b.state(kb)
    assert torch.equal(ka, kb)


def test_hit_target(oracle_mod, tiny):
    from paper_2606_28372_b300 import catune as ct
    tgt = np.float32(1.01 * float(tiny.table.min()))
    E = oracle_mod.run("de", tiny.osp, tiny.okeys, tiny.table, pop=20, gens=100, seed=0, target=tgt)
    o = ct.Opt(tiny.sp, "de", 20, 0, target=tgt)
    for g in range(101):
        o.step(g)
    b = o.best()
    assert (b["hit_gen"], b["hit_evals"]) == (int(E["hit"][0]), int(E["hit"][1]))
