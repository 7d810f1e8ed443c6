"""GPU parity of the paper's repair rules (index distance for DE, Algorithms 2 and 3) and of
whole optimizer runs that use them."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64, to_dev_u64
from tests.test_gpu_optim import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spaces(oracle_mod):
    return {n: Pair(sd, oracle_mod) for n, sd in (("tiny", W.tiny_space()), ("medium", W.medium_space()),
                                                   ("b9", W.batched_space(9)))}


@pytest.mark.parametrize("name", ["tiny", "medium", "b9"])
@pytest.mark.parametrize("rule", [1, 2, 3])
@pytest.mark.parametrize("lut", [False, True])
def test_repair_paper_matches_oracle(oracle_mod, spaces, name, rule, lut, monkeypatch):
    """Both forms of the scan: the per-field loop and the per-candidate tables (forced on these
    short slices by lowering the slice threshold)."""
    if lut:
        monkeypatch.setenv("CATUNE_RULE_LUT_MIN_SLICE", "1")
    p = spaces[name]
    sd, O = p.sd, oracle_mod
    n = 150
    base = O.unpack(p.osp, p.okeys[W.random_ranks(len(p.okeys), n // 3, seed=rule)])
    cand = np.concatenate([O.pack(p.osp, W.uniform_tuples(sd, n // 3, seed=rule)),
                           O.pack(p.osp, W.perturbed_tuples(sd, base, seed=rule)),
                           p.okeys[W.random_ranks(len(p.okeys), n - 2 * (n // 3), seed=rule + 7)]])
    r = np.array(sd.n_values)
    eps = np.float32(1.0 / (r.max() - 1))
    rng = np.random.default_rng(rule)
    pos = np.clip(O.unpack(p.osp, cand) * eps + rng.normal(scale=0.6 * eps, size=(len(cand), len(r))), 0, 1).astype(np.float32)
    words = rng.integers(0, 2 ** 32, len(cand), dtype=np.uint64).astype(np.uint32)
    exp = O.repair_paper(rule, p.osp, p.okeys, cand, pos=pos, eps=eps, words=words)
    out = torch.empty(len(cand), dtype=torch.int64, device="cuda")
    p.sp.repair_paper(rule, to_dev_u64(cand), out, pos=torch.from_numpy(pos).cuda(), eps=float(eps),
                      words=torch.from_numpy(words.view(np.int32)).cuda())
    assert np.array_equal(from_dev_u64(out), exp)


def step_trace(p, kind, pop, gens, seed, **params):
    """Whole generations through ct_opt_step (the run's own repair rule), read back per generation."""
    from paper_2606_28372_b300 import catune as ct
    o = ct.Opt(p.sp, kind, pop, seed, **params)
    n = len(p.sd.params)
    b = [torch.empty(pop, dtype=torch.int64, device="cuda") for _ in range(3)]
    fit = torch.empty(pop, dtype=torch.float32, device="cuda")
    popf = torch.empty(pop, dtype=torch.float32, device="cuda")
    pos = torch.empty(pop * n, dtype=torch.float32, device="cuda")
    T = {k: [] for k in ("cand", "evalk", "fit", "popk", "popf", "pos", "best_key", "best_fit", "n_unique")}
    for g in range(gens + 1):
        o.step(g)
        o.last_generation(b[0], None, b[1], fit)
        o.state(b[2], popf, pos)
        T["cand"].append(from_dev_u64(b[0]))
        T["evalk"].append(from_dev_u64(b[1]))
        T["fit"].append(fit.cpu().numpy())
        T["popk"].append(from_dev_u64(b[2]))
        T["popf"].append(popf.cpu().numpy())
        T["pos"].append(pos.cpu().numpy().reshape(pop, n))
        bb = o.best()
        T["best_key"].append(bb["best_key"])
        T["best_fit"].append(np.float32(bb["best_fit"]))
        T["n_unique"].append(bb["n_unique"])
    return {k: np.array(v) for k, v in T.items()}


@pytest.mark.parametrize("kind", ["de", "pso", "firefly", "ga"])
@pytest.mark.parametrize("name,pop,gens", [("tiny", 20, 30), ("medium", 64, 8)])
def test_trajectory_with_paper_rules(oracle_mod, spaces, kind, name, pop, gens):
    p = spaces[name]
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=pop, gens=gens, seed=4, repair_rule=1)
    T = step_trace(p, kind, pop, gens, 4, repair_rule=1)
    for f in ("cand", "evalk", "fit", "popk", "popf", "best_key", "best_fit", "n_unique") + (("pos",) if kind in ("pso", "firefly") else ()):
        a, b = T[f], E[f].astype(T[f].dtype)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{f} differs first at {bad[0]} ({len(bad)} entries)")
    # the rule changes the run: some evaluated configuration differs from the Hamming rule's
    H = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=pop, gens=gens, seed=4)
    assert not np.array_equal(H["evalk"], E["evalk"])


@pytest.mark.parametrize("kind", ["de", "pso", "ga"])
def test_trajectory_with_paper_rules_tables(oracle_mod, spaces, kind, monkeypatch):
    monkeypatch.setenv("CATUNE_RULE_LUT_MIN_SLICE", "1")
    p = spaces["medium"]
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=48, gens=8, seed=5, repair_rule=1)
    T = step_trace(p, kind, 48, 8, 5, repair_rule=1)
    for f in ("cand", "evalk", "fit", "popk", "best_key", "n_unique"):
        assert np.array_equal(T[f], E[f].astype(T[f].dtype)), f


def test_repair_paper_tables_at_size(oracle_mod):
    """A 26.8M-key space: long enough slices that the table form runs by default."""
    sd = W._space("wide", [(f"p{k}", list(range(8))) for k in range(8)] + [("q", [0, 1])], ["p0 + p1 <= 12"])
    p = Pair(sd, oracle_mod, table=None)
    assert len(p.okeys) > 20_000_000
    n = 12
    base = oracle_mod.unpack(p.osp, p.okeys[W.random_ranks(len(p.okeys), n, seed=3)])
    cand = oracle_mod.pack(p.osp, np.clip(base + np.array([[7, 7] + [0] * 7]), 0, 7))   # p0 + p1 > 12
    r = np.array(sd.n_values)
    eps = np.float32(1.0 / (r.max() - 1))
    rng = np.random.default_rng(4)
    pos = np.clip(oracle_mod.unpack(p.osp, cand) * eps + rng.normal(scale=0.6 * eps, size=(n, len(r))), 0, 1).astype(np.float32)
    words = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    for rule in (1, 2, 3):
        exp = oracle_mod.repair_paper(rule, p.osp, p.okeys, cand, pos=pos, eps=eps, words=words)
        out = torch.empty(n, dtype=torch.int64, device="cuda")
        p.sp.repair_paper(rule, to_dev_u64(cand), out, pos=torch.from_numpy(pos).cuda(), eps=float(eps),
                          words=torch.from_numpy(words.view(np.int32)).cuda())
        assert np.array_equal(from_dev_u64(out), exp), rule


@pytest.mark.parametrize("kind", ["de", "ga", "pso"])
def test_graph_with_paper_rules(oracle_mod, spaces, kind):
    from paper_2606_28372_b300 import catune as ct
    p = spaces["medium"]
    E = oracle_mod.run(kind, p.osp, p.okeys, p.table, pop=32, gens=6, seed=9, repair_rule=1)
    o = ct.Opt(p.sp, kind, 32, 9, repair_rule=1)
    o.run_graph(0, 1)
    o.run_graph(1, 6)
    k = torch.empty(32, dtype=torch.int64, device="cuda")
    o.state(k)
    assert np.array_equal(from_dev_u64(k), E["popk"][6])
    assert o.best()["n_unique"] == int(E["n_unique"][6])
