"""Pins of the oracle's paper-faithful repairs (Section IV-A neighbour rules, Algorithm 1's
index-distance repair, Algorithms 2 and 3), against numpy restatements of the set definitions."""
import numpy as np
import pytest

from paper_2606_28372_b300 import workloads as W


@pytest.fixture(scope="module")
def med(oracle_mod):
    sd = W.medium_space()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    return sd, sp, keys, oracle_mod.unpack(sp, keys)


def _cands(O, sd, sp, keys, n, seed):
    c = O.pack(sp, W.uniform_tuples(sd, 4 * n, seed=seed))
    return np.setdiff1d(c, keys)[:n]


def test_index_distance_repair(oracle_mod, med):
    sd, sp, keys, V = med
    c = _cands(oracle_mod, sd, sp, keys, 40, 1)
    out = oracle_mod.repair_paper(1, sp, keys, c)
    for u, k in zip(oracle_mod.unpack(sp, c), out):
        d = np.abs(V - u).sum(axis=1)
        assert k == keys[np.flatnonzero(d == d.min())[0]]          # smallest key among the L1-nearest
    valid = oracle_mod.repair_paper(1, sp, keys, keys[:50])
    assert np.array_equal(valid, keys[:50])


def test_adjacent_rule_skips_values_absent_from_the_space(oracle_mod, med):
    """by = 64 occurs in no valid configuration of the medium space (by*ty <= 16), so from by = 64
    the adjacent rule steps to by = 16 while strictly adjacent would need by = 32."""
    sd, sp, keys, V = med
    r = np.array(sd.n_values)
    occ = [np.isin(np.arange(r[k]), np.unique(V[:, k])) for k in range(len(r))]
    assert not occ[1][6] and occ[1][4]
    u = np.array([0, 6, 0, 0, 2, 0, 1, 0, 1, 0])
    sa, adj, ham = _sets(u, V, occ)
    assert not sa.any() and adj.any() and (V[adj][:, 1] == 4).all()


def _sets(u, V, occ):
    d = V - u
    nz = d != 0
    sa = (np.abs(d) <= 1).all(axis=1) & nz.any(axis=1)
    lo = np.array([max([t for t in range(u[k]) if occ[k][t]], default=-1) for k in range(len(u))])
    hi = np.array([min([t for t in range(u[k] + 1, len(occ[k])) if occ[k][t]], default=-1) for k in range(len(u))])
    adj = ((~nz) | (V == lo) | (V == hi)).all(axis=1) & nz.any(axis=1)
    ham = nz.sum(axis=1) == 1
    return [sa, adj, ham]


def test_algorithm2_first_nonempty_set_and_closest(oracle_mod, med):
    sd, sp, keys, V = med
    r = np.array(sd.n_values)
    occ = [np.isin(np.arange(r[k]), np.unique(V[:, k])) for k in range(len(r))]
    c = _cands(oracle_mod, sd, sp, keys, 30, 2)
    eps = np.float32(1.0 / (r.max() - 1))
    rng = np.random.default_rng(3)
    pos = np.clip(oracle_mod.unpack(sp, c) * eps + rng.normal(scale=0.4 * eps, size=(len(c), len(r))), 0, 1).astype(np.float32)
    out = oracle_mod.repair_paper(2, sp, keys, c, pos=pos, eps=eps)
    ham, _ = oracle_mod.repair(sp, keys, c)
    used = [0, 0, 0, 0]
    for u, x, k, h in zip(oracle_mod.unpack(sp, c), pos, out, ham):
        sets = _sets(u, V, occ)
        which = next((i for i, s in enumerate(sets) if s.any()), 3)
        used[which] += 1
        if which == 3:                         # no neighbour in any set: nearest valid (Hamming)
            assert k == h
            continue
        first = sets[which]
        rk = np.searchsorted(keys, k)
        assert keys[rk] == k and first[rk]
        dist = ((V[first] * np.float64(eps) - x) ** 2).sum(axis=1)
        assert dist.min() >= ((V[rk] * np.float64(eps) - x) ** 2).sum() - 1e-6
    assert used[0] and used[3]


def test_algorithm3_random_member(oracle_mod, med):
    sd, sp, keys, V = med
    r = np.array(sd.n_values)
    occ = [np.isin(np.arange(r[k]), np.unique(V[:, k])) for k in range(len(r))]
    cs = _cands(oracle_mod, sd, sp, keys, 30, 4)
    c = next(x for x in cs if any(s.any() for s in _sets(oracle_mod.unpack(sp, [x])[0], V, occ)))
    c = np.array([c], np.uint64)
    u = oracle_mod.unpack(sp, c)[0]
    first = next(s for s in _sets(u, V, occ) if s.any())
    members = keys[first]
    words = np.random.default_rng(5).integers(0, 2 ** 32, 4000, dtype=np.uint64).astype(np.uint32)
    out = oracle_mod.repair_paper(3, sp, keys, np.repeat(c, len(words)), words=words)
    assert np.isin(out, members).all()
    freq = np.array([np.sum(out == m) for m in members]) / len(out)
    assert np.abs(freq - 1.0 / len(members)).max() < 4.0 / np.sqrt(len(out)) + 0.02
