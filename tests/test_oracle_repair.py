"""Pins of the oracle's lookup and nearest-valid repair (Section IV-A neighbours, Algorithm 1
Repair), using an evaluator independent of the oracle: Python's own integer expressions."""
import itertools

import numpy as np
import pytest

from paper_2606_28372_b300 import workloads as W
from tests.test_oracle_space import py_valid


def _ball(u, r, d):
    """All tuples at Hamming distance exactly d from u."""
    n = len(u)
    for S in itertools.combinations(range(n), d):
        for alt in itertools.product(*[[v for v in range(r[k]) if v != u[k]] for k in S]):
            t = list(u)
            for k, v in zip(S, alt):
                t[k] = v
            yield t


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_repair_minimal_by_independent_ball(oracle_mod, name):
    sd = W.SPACES[name]()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    cands = np.concatenate([W.uniform_tuples(sd, 12, seed=11),
                            W.perturbed_tuples(sd, oracle_mod.unpack(sp, keys[::max(1, len(keys) // 12)][:12]), seed=5)])
    ck = oracle_mod.pack(sp, cands)
    rep, dist = oracle_mod.repair(sp, keys, ck)
    r = sd.n_values
    for u, k, d in zip(cands, rep, dist):
        v = oracle_mod.unpack(sp, [k])[0]
        assert py_valid(sd, v)                                    # repaired is valid
        assert int(np.sum(v != u)) == d                          # reported distance is real
        for dd in range(d):                                       # nothing valid closer
            assert not any(py_valid(sd, t) for t in _ball(list(u), r, dd))
        # no valid point at distance d with a smaller key
        for t in _ball(list(u), r, d):
            kt = int(oracle_mod.pack(sp, [t])[0])
            if kt < int(k):
                assert not py_valid(sd, t)


def test_repair_identity_on_valid_and_lookup(oracle_mod):
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    pick = keys[W.random_ranks(len(keys), 200, seed=2)]
    rep, dist = oracle_mod.repair(sp, keys, pick)
    assert np.array_equal(rep, pick) and not dist.any()
    rk = oracle_mod.lookup(keys, pick)
    assert np.array_equal(rk, np.searchsorted(keys, pick))
    bad = oracle_mod.pack(sp, W.uniform_tuples(sd, 500, seed=4))
    rk = oracle_mod.lookup(keys, bad)
    inset = np.isin(bad, keys)
    assert np.array_equal(rk >= 0, inset)


def test_repair_rejects_out_of_domain(oracle_mod):
    sp = oracle_mod.from_def(W.tiny_space())
    keys = oracle_mod.valid_keys(sp)
    with pytest.raises(ValueError):
        oracle_mod.repair(sp, keys, np.array([6], dtype=np.uint64))       # unroll index 6 of 6
    with pytest.raises(ValueError):
        oracle_mod.repair(sp, keys, np.array([1 << 12], dtype=np.uint64))  # above key width
