"""Parity at the benchmarked sizes: the medium workload (all four optimizers, pop 128, 500
generations) generation by generation against the oracle, and the batched workload (4,096 runs
over the 32 batched spaces, 100 generations, autotuned launch shape, one CUDA graph) on sampled
runs against the same runs done alone and against the oracle."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64
from tests.test_gpu_rules import step_trace

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
def test_medium_full_size_trajectory(oracle_mod, kind):
    p = Pair(W.medium_space(), oracle_mod)
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=128, gens=499, seed=0)
    T = step_trace(p, kind, 128, 499, 0)
    for f in ("cand", "evalk", "fit", "popk", "popf", "best_key", "best_fit", "n_unique"):
        a, b = T[f], E[f].astype(T[f].dtype)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{f} differs first at {bad[0]} ({len(bad)} entries)")


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
def test_medium_full_size_more_seeds(oracle_mod, kind):
    """Seeds 1, 2 and 3 of the same workload at full length.  The oracle runs of the three seeds
    go to threads (the oracle's C calls release the interpreter lock), the GPU runs one by one."""
    from concurrent.futures import ThreadPoolExecutor
    p = Pair(W.medium_space(), oracle_mod)
    seeds = (1, 2, 3)
    with ThreadPoolExecutor(len(seeds)) as ex:
        futs = {s: ex.submit(oracle_mod.run, kind, p.osp, p.okeys, p.table, 128, 499, s) for s in seeds}
        traces = {s: step_trace(p, kind, 128, 499, s) for s in seeds}
        for s in seeds:
            E, T = futs[s].result(), traces[s]
            for f in ("cand", "evalk", "fit", "popk", "popf", "best_key", "best_fit", "n_unique"):
                a, b = T[f], E[f].astype(T[f].dtype)
                if not np.array_equal(a, b):
                    bad = np.argwhere(a != b)
                    raise AssertionError(f"seed {s}: {f} differs first at {bad[0]} ({len(bad)} entries)")


def test_batched_full_size(oracle_mod, tmp_path):
    from paper_2606_28372_b300 import catune as ct
    dev = torch.device("cuda", 0)
    spaces, tables = [], []
    for si in range(32):                               # built as the benchmark builds them
        sd = W.batched_space(si)
        sp = ct.Space.from_def(sd)
        sp.build()
        t = W.smooth_table(sd, sp.unpack(from_dev_u64(sp.keys())), seed=si)
        sp._t = torch.from_numpy(t).to(dev)
        sp.set_fitness(sp._t)
        spaces.append(sp)
        tables.append(t)
    kinds = ["de", "pso", "ga"]
    runs = [(r % 32, kinds[r % 3], 32 * (1 + (r // 3) % 4), r, float(np.float32(1.01 * tables[r % 32].min())))
            for r in range(4096)]
    gens = 100
    b = ct.Batch(spaces, runs)
    b.autotune(str(tmp_path / "tune.jsonl"), gens=3)
    b.run_graph(gens)
    res = b.results()
    for r in [0, 1, 2, 37, 100, 515, 1024, 2047, 2900, 3333, 4000, 4095]:
        si, kind, pop, seed, tgt = runs[r]
        o = ct.Opt(spaces[si], kind, pop, seed, target=tgt)
        o.run_graph(0, 1)
        o.run_graph(1, gens - 1)
        ka, kb = (torch.empty(pop, dtype=torch.int64, device=dev) for _ in range(2))
        fa, fb = (torch.empty(pop, dtype=torch.float32, device=dev) for _ in range(2))
        b.run_state(r, ka, fa)
        o.state(kb, fb)
        assert torch.equal(ka, kb) and torch.equal(fa, fb), r
        sb = o.best()
        assert int(res["best_key"][r]) == sb["best_key"] and int(res["n_unique"][r]) == sb["n_unique"], r
        assert int(res["hit_evals"][r]) == sb["hit_evals"], r
    for r in (0, 3, 6, 129):                             # spaces 0, 3, 6, 1: small enough for the oracle
        si, kind, pop, seed, tgt = runs[r]
        q = Pair(W.batched_space(si), oracle_mod, table="smooth", seed=si)
        assert np.array_equal(q.table, tables[si])
        E = oracle_mod.run(kind, q.osp, q.okeys, q.table, pop=pop, gens=gens - 1, seed=seed, target=tgt)
        k = torch.empty(pop, dtype=torch.int64, device=dev)
        b.run_state(r, k)
        assert np.array_equal(from_dev_u64(k), E["popk"][-1]), r
        assert int(res["n_unique"][r]) == int(E["n_unique"][-1]) and int(res["hit_evals"][r]) == int(E["hit"][1]), r


def test_surrogate_on_the_large_space():
    """The surrogate at the large size (pop 256, a pool of 4,096 repaired candidates per screened
    generation).  A generation the judge does not screen proposes exactly what the plain run
    proposes, so up to the first screened generation the two trajectories are equal; a forced
    screen must then choose every slot's key from its own pool of repaired candidates."""
    from paper_2606_28372_b300 import catune as ct
    dev = torch.device("cuda", 0)
    sd = W.large_space()
    sp = ct.Space.from_def(sd)
    nv = sp.build()
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    table = torch.exp(torch.randn(nv, generator=g, device=dev, dtype=torch.float32))
    sp.set_fitness(table)
    logt = torch.log(table)
    P, G = 256, 10
    plain = ct.Opt(sp, "de", P, 3)
    surr = ct.Opt(sp, "de", P, 3)
    surr.set_surrogate(logt)
    kp, ks = (torch.empty(P, dtype=torch.int64, device=dev) for _ in range(2))
    opened = None
    for gen in range(G + 1):
        plain.step(gen)
        surr.step(gen)
        info = surr.surrogate_info()
        if info["screened"] and opened is None:
            opened = gen
        if opened is None:
            plain.state(kp)
            surr.state(ks)
            assert torch.equal(kp, ks), gen
            assert plain.best() == surr.best(), gen
    forced = ct.Opt(sp, "de", P, 4)
    forced.set_surrogate(logt, warmup_mult=0, mae_ratio=1e30)
    rep = torch.empty(P, dtype=torch.int64, device=dev)
    rank = torch.empty(P, dtype=torch.int64, device=dev)
    for gen in range(4):
        forced.step(gen)
        forced.last_generation(None, rep)
        sp.lookup(rep, rank)
        assert bool((rank >= 0).all()), gen                    # chosen candidates are repaired
    assert forced.surrogate_info()["screened"]
