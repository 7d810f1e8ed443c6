"""GPU parity: lookup, nearest-valid repair and evaluation against the oracle."""
import itertools

import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64, to_dev_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pairs(oracle_mod):
    return {n: Pair(W.SPACES[n](), oracle_mod) for n in ("tiny", "medium")}


def _cands(p, seed, count=600):
    sd, O = p.sd, p.O
    base = O.unpack(p.osp, p.okeys[W.random_ranks(len(p.okeys), count // 3, seed)])
    return np.concatenate([
        O.pack(p.osp, W.uniform_tuples(sd, count // 3, seed)),
        O.pack(p.osp, W.perturbed_tuples(sd, base, seed)),
        p.okeys[W.random_ranks(len(p.okeys), count - 2 * (count // 3), seed + 1)],
    ])


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_lookup(pairs, name):
    p = pairs[name]
    c = _cands(p, 3)
    rank = torch.empty(len(c), dtype=torch.int64, device="cuda")
    p.sp.lookup(to_dev_u64(c), rank)
    assert np.array_equal(rank.cpu().numpy(), p.O.lookup(p.okeys, c))


@pytest.mark.parametrize("name", ["tiny", "medium"])
@pytest.mark.parametrize("mode,radius", [(0, 0), (1, 0), (2, 1), (2, 2), (2, 3)])
def test_repair(pairs, name, mode, radius):
    p = pairs[name]
    c = _cands(p, 5 + mode + radius)
    p.sp.set_repair_mode(mode, radius)
    out = torch.empty(len(c), dtype=torch.int64, device="cuda")
    dist = torch.empty(len(c), dtype=torch.uint8, device="cuda")
    p.sp.repair(to_dev_u64(c), out, dist)
    eo, ed = p.O.repair(p.osp, p.okeys, c)
    p.sp.set_repair_mode(0, 0)
    assert np.array_equal(from_dev_u64(out), eo)
    assert np.array_equal(dist.cpu().numpy(), ed)


def test_repair_ragged_and_empty(pairs):
    p = pairs["medium"]
    for n in (0, 1, 31, 33, 1000):
        c = _cands(p, 40 + n, count=max(n, 3))[:n]
        out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")[:n]
        p.sp.repair(to_dev_u64(c) if n else torch.empty(0, dtype=torch.int64, device="cuda"), out)
        if n:
            assert np.array_equal(from_dev_u64(out), p.O.repair(p.osp, p.okeys, c)[0])


def test_repair_bad_candidate_status(pairs):
    from paper_2606_28372_b300 import catune as ct
    p = pairs["tiny"]
    c = np.array([p.okeys[0], 6, 1 << 12], dtype=np.uint64)   # unroll index 6 of 6; bit above the key
    out = torch.empty(3, dtype=torch.int64, device="cuda")
    dist = torch.empty(3, dtype=torch.uint8, device="cuda")
    p.sp.repair(to_dev_u64(c), out, dist)
    assert p.sp.status() == ct.CT_ERR_INVALID_ARG
    assert list(dist.cpu().numpy()) == [0, 255, 255]
    assert p.sp.status() == ct.CT_OK


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_evaluate(pairs, name):
    p = pairs[name]
    c = _cands(p, 9)
    fit = torch.empty(len(c), dtype=torch.float32, device="cuda")
    rank = torch.empty(len(c), dtype=torch.int64, device="cuda")
    p.sp.evaluate(to_dev_u64(c), fit, rank)
    r = p.O.lookup(p.okeys, c)
    want = np.where(r >= 0, p.table[np.maximum(r, 0)], np.float32(np.inf))
    assert np.array_equal(rank.cpu().numpy(), r)
    assert np.array_equal(fit.cpu().numpy(), want)


def test_large_repair_properties(oracle_mod):
    """Full-size large space: every repaired candidate is valid, its distance is real, and no
    valid point is closer or equally close with a smaller key (checked by the oracle's
    constraint evaluator over the Hamming balls)."""
    from paper_2606_28372_b300 import catune as ct
    sd = W.large_space()
    sp = ct.Space.from_def(sd)
    sp.build()
    osp = oracle_mod.from_def(sd)
    keys = sp.keys()
    base_rank = W.random_ranks(695_228_960, 64, seed=2)
    base = sp.unpack(from_dev_u64(keys[torch.from_numpy(base_rank).cuda()]))
    cand = np.concatenate([oracle_mod.pack(osp, W.uniform_tuples(sd, 64, seed=4)),
                           oracle_mod.pack(osp, W.perturbed_tuples(sd, base, seed=4))])
    out = torch.empty(len(cand), dtype=torch.int64, device="cuda")
    dist = torch.empty(len(cand), dtype=torch.uint8, device="cuda")
    sp.repair(to_dev_u64(cand), out, dist)
    o, d = from_dev_u64(out), dist.cpu().numpy()
    r = sd.n_values
    assert oracle_mod.check_tuples(osp, oracle_mod.unpack(osp, o)).all()
    checked = 0
    for u, k, dd in zip(oracle_mod.unpack(osp, cand), o, d):
        v = oracle_mod.unpack(osp, [k])[0]
        assert int(np.sum(u != v)) == dd
        if dd > 3:
            continue
        for rad in range(dd + 1):
            pts = []
            for S in itertools.combinations(range(16), rad):
                for alt in itertools.product(*[[x for x in range(r[q]) if x != u[q]] for q in S]):
                    t = u.copy()
                    t[list(S)] = alt
                    pts.append(t)
            if not pts:
                continue
            pts = np.array(pts)
            ok = oracle_mod.check_tuples(osp, pts)
            if rad < dd:
                assert not ok.any()
            else:
                pk = oracle_mod.pack(osp, pts[ok])
                assert pk.min() == k
        checked += 1
    assert checked >= 64


@pytest.fixture(scope="module")
def scan_spaces(oracle_mod):
    """Spaces with keys narrower and wider than 32 bits and with even and odd |V|."""
    from paper_2606_28372_b300 import catune as ct
    defs = [W.tiny_space(), W.batched_space(3),
            W._space("wide33_odd", [(f"p{i}", range(1, 6)) for i in range(11)], ["(p0*p1 + p2*p3 + p4) % 17 == 2"])]
    out = []
    for sd in defs:
        osp = oracle_mod.from_def(sd)
        okeys = oracle_mod.valid_keys(osp)
        sp = ct.Space.from_def(sd)
        assert sp.build() == len(okeys)
        out.append((sd, osp, okeys, sp))
    assert len(out[2][2]) % 2 == 1 and out[2][3].info().key_bits == 33
    return out


@pytest.mark.parametrize("count", [1, 2, 3, 4, 5, 9, 17, 33, 70])
def test_scan_widths_and_odd_tail(oracle_mod, scan_spaces, count):
    """Scan-only repair for every pending-candidate width."""
    for sd, osp, okeys, sp in scan_spaces:
        inv = np.setdiff1d(oracle_mod.pack(osp, W.uniform_tuples(sd, 4 * count + 40, seed=count)), okeys)[:count]
        assert len(inv) == count
        sp.set_repair_mode(1, 0)
        out = torch.empty(count, dtype=torch.int64, device="cuda")
        dist = torch.empty(count, dtype=torch.uint8, device="cuda")
        sp.repair(to_dev_u64(inv), out, dist)
        sp.set_repair_mode(0, 0)
        eo, ed = oracle_mod.repair(osp, okeys, inv)
        assert np.array_equal(from_dev_u64(out), eo), sd.name
        assert np.array_equal(dist.cpu().numpy(), ed), sd.name
