"""Pins of the oracle's search-space construction (Section IV-A) against facts outside it."""
import itertools
import os

import numpy as np
import pytest

from paper_2606_28372_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def py_valid(sd, idx):
    """Independent evaluator: Python's own integers and operators (all operands here are
    non-negative, so floor division equals the truncating division of the spec)."""
    env = {n: sd.values[k][i] for k, (n, i) in enumerate(zip(sd.names, idx))}
    return all(bool(eval(c, {"__builtins__": {}, "min": min, "max": max}, env))
               for c in sd.constraints)


def test_tiny_hand_count(oracle_mod):
    lines = [l.split() for l in open(os.path.join(GOLD, "tiny_hand_count.txt"))
             if l.strip() and not l.startswith("#")]
    total = int([l for l in lines if l[0] == "TOTAL"][0][1])
    rows = [l for l in lines if l[0] != "TOTAL"]
    assert sum(int(r[3]) for r in rows) * 6 == total == 732
    sp = oracle_mod.from_def(W.tiny_space())
    keys = oracle_mod.valid_keys(sp)
    assert len(keys) == total
    # per-bx breakdown matches the hand count
    idx = oracle_mod.unpack(sp, keys)
    for k, r in enumerate(rows):
        assert int(np.sum(idx[:, 0] == k)) == int(r[3]) * 6


@pytest.mark.parametrize("name", ["large_a", "large_b", "tiny"])
def test_group_brute_force_independent_evaluator(oracle_mod, name):
    sd = W.SPACES[name]()
    cnt = sum(py_valid(sd, idx) for idx in itertools.product(*[range(r) for r in sd.n_values]))
    sp = oracle_mod.from_def(sd)
    assert oracle_mod.enumerate_range(sp, count_only=True) == cnt


def test_medium_factorised_count(oracle_mod):
    """Count the medium space by factorising the free parameters (unroll, splitk, ro), with
    Python integers; compare with the oracle's brute force."""
    sd = W.medium_space()
    v = dict(zip(sd.names, sd.values))
    total = 0
    for bx, by, tx, ty, vec, pad, st in itertools.product(v["bx"], v["by"], v["tx"], v["ty"],
                                                          v["vec"], v["pad"], v["stages"]):
        if not (64 <= bx * by <= 1024 and bx % (tx * vec) == 0 and by * ty <= 16
                and 4 * (bx * tx + pad) * (by * ty) * st <= 49152 and vec * tx <= 8):
            continue
        n_unroll = sum(1 for u in v["unroll"] if u * vec <= tx * ty)
        n_split = sum(1 for s in v["splitk"] if s <= 2 or st >= 4)
        n_ro = sum(1 for r in v["ro"] if r == 0 or pad == 0)
        total += n_unroll * n_split * n_ro
    sp = oracle_mod.from_def(sd)
    assert oracle_mod.enumerate_range(sp, count_only=True) == total == 139604


def test_large_closed_form_and_window(oracle_mod):
    """|V(large)| = |V(A)| * |V(B)|, and any Cartesian window of the large space holds exactly
    the (A-valid, B-valid) pairs of that window."""
    a = oracle_mod.valid_keys(oracle_mod.from_def(W.large_group_a()))
    b = oracle_mod.valid_keys(oracle_mod.from_def(W.large_group_b()))
    assert len(a) * len(b) == 695_228_960
    sd = W.large_space()
    sp = oracle_mod.from_def(sd)
    _, _, bits_b = oracle_mod.key_layout(oracle_mod.from_def(W.large_group_b()))
    nb = W.large_group_b().cartesian_size
    for c0 in (0, 25_000_123_456, sd.cartesian_size - 600_000):
        c1 = min(sd.cartesian_size, c0 + 600_000)
        got = oracle_mod.enumerate_range(sp, c0, c1)
        # expected from the groups: Cartesian c = ca * |B| + cb
        aset = set(int(x) for x in a)
        bset = set(int(x) for x in b)
        exp = []
        sa, sb = oracle_mod.from_def(W.large_group_a()), oracle_mod.from_def(W.large_group_b())
        for ca in range(c0 // nb, (c1 - 1) // nb + 1):
            ka = oracle_mod.enumerate_range(sa, ca, ca + 1)
            if len(ka) == 0:
                continue
            lo, hi = max(c0 - ca * nb, 0), min(c1 - ca * nb, nb)
            kb = oracle_mod.enumerate_range(sb, lo, hi)
            exp.extend((int(ka[0]) << bits_b) | int(x) for x in kb)
        assert [int(x) for x in got] == exp
        assert all(int(x) >> bits_b in aset and int(x) & ((1 << bits_b) - 1) in bset for x in got)


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_keys_sorted_and_valid(oracle_mod, name):
    sd = W.SPACES[name]()
    sp = oracle_mod.from_def(sd)
    keys = oracle_mod.valid_keys(sp)
    assert np.all(keys[1:] > keys[:-1])
    idx = oracle_mod.unpack(sp, keys)
    rng = np.random.default_rng(7)
    for row in idx[rng.integers(0, len(idx), 300)]:
        assert py_valid(sd, row)
    # points outside V are invalid under the independent evaluator
    allt = W.uniform_tuples(sd, 2000, seed=3)
    ok = oracle_mod.check_tuples(sp, allt)
    for row, o in zip(allt, ok):
        assert o == py_valid(sd, row)
    kset = set(int(k) for k in keys)
    for row, o in zip(allt, ok):
        assert (int(oracle_mod.pack(sp, row[None])[0]) in kset) == o


def test_key_layout_closed_form(oracle_mod):
    sp = oracle_mod.from_def(W.large_space())
    w, o, bits = oracle_mod.key_layout(sp)
    r = W.large_space().n_values
    assert list(w) == [int(np.ceil(np.log2(x))) for x in r]
    assert bits == 40 and o[-1] == 0 and all(o[k] == o[k + 1] + w[k + 1] for k in range(15))
    assert oracle_mod.key_layout(oracle_mod.from_def(W.medium_space()))[2] == 26
    assert oracle_mod.key_layout(oracle_mod.from_def(W.tiny_space()))[2] == 12


def test_no_constraints_and_contradiction(oracle_mod):
    vals = [[1, 2, 3], [5, 6], [7, 8, 9, 10, 11]]
    sp = oracle_mod.make_space(["a", "b", "c"], vals, [])
    keys = oracle_mod.valid_keys(sp)
    assert len(keys) == 30
    idx = oracle_mod.unpack(sp, keys)
    assert [tuple(r) for r in idx] == list(itertools.product(range(3), range(2), range(5)))
    sp2 = oracle_mod.make_space(["a", "b", "c"], vals, ["a<0"])
    assert len(oracle_mod.valid_keys(sp2)) == 0


def test_expression_semantics(oracle_mod):
    """Truncating division/modulo, poison on division by zero, chained comparisons."""
    vals = [[-7, -1, 0, 3, 7], [-2, 0, 2, 3]]
    names = ["a", "b"]
    cases = {
        "a//b == -3": lambda a, b: b != 0 and int(a / b) == -3,
        "a%b == -1": lambda a, b: b != 0 and a - b * int(a / b) == -1,
        "b==0 or a//b>=1": lambda a, b: b == 0 or int(a / b) >= 1,
        "not (a//b > 0)": lambda a, b: b == 0 or not int(a / b) > 0,
        "-2 <= a*b < 6": lambda a, b: -2 <= a * b < 6,
        "min(a, b) + max(a, 1) == 0": lambda a, b: min(a, b) + max(a, 1) == 0,
    }
    for expr, ref in cases.items():
        sp = oracle_mod.make_space(names, vals, [expr])
        tuples = np.array(list(itertools.product(range(5), range(4))))
        got = oracle_mod.check_tuples(sp, tuples)
        want = [ref(vals[0][i], vals[1][j]) for i, j in tuples]
        assert list(got) == want, expr
