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


def _ball_path(path, monkeypatch):
    """near: the default (table test and small radii in one launch); point: every radius by the
    per-point kernel; filtered: every radius by the filtered warp-per-subset kernel."""
    if path in ("point", "filtered"):
        monkeypatch.setenv("CATUNE_BALL_NEAR_POINTS", "0")
    if path == "filtered":
        monkeypatch.setenv("CATUNE_BALL_FS_MIN_AVG", "0")


@pytest.mark.parametrize("path", ["near", "point", "filtered"])
@pytest.mark.parametrize("name", ["tiny", "medium"])
@pytest.mark.parametrize("mode,radius", [(0, 0), (1, 0), (2, 1), (2, 2), (2, 3)])
def test_repair(pairs, name, mode, radius, path, monkeypatch):
    """Every repair mode against the oracle, by each path of the ball search."""
    if path != "near" and mode == 1:
        pytest.skip("no ball search")
    _ball_path(path, monkeypatch)
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
            W._space("wide33_odd", [(f"p{i}", range(1, 6)) for i in range(11)], ["(p0*p1 + p2*p3 + p4) % 17 == 2"]),
            # single-value parameters (fields of zero bits) between the others
            W._space("zero_width", [("a", range(7)), ("z0", [3]), ("b", range(5)), ("c", range(6)), ("z1", [1]),
                                    ("d", range(9)), ("e", range(3))], ["(a + 2*b + c*d + e) % 5 != 1", "a*e <= 8"]),
            # a 9-bit parameter: no table plan, the SWAR scan runs either way
            W._space("wide_field", [("a", range(300)), ("b", range(5)), ("c", range(4))], ["(a*b + c) % 7 == 3"])]
    out = []
    for sd in defs:
        osp = oracle_mod.from_def(sd)
        okeys = oracle_mod.valid_keys(osp)
        sp = ct.Space.from_def(sd)
        assert sp.build() == len(okeys)
        out.append((sd, osp, okeys, sp))
    assert len(out[2][2]) % 2 == 1 and out[2][3].info().key_bits == 33
    return out


@pytest.mark.parametrize("lut", [False, True])
@pytest.mark.parametrize("count", [1, 2, 3, 4, 5, 9, 17, 33, 45, 70])
def test_scan_widths_and_odd_tail(oracle_mod, scan_spaces, count, lut, monkeypatch):
    """Scan-only repair for every pending-candidate width, with the SWAR distance and with the
    per-candidate distance tables (forced on short key arrays)."""
    monkeypatch.setenv("CATUNE_SCAN_LUT_MIN_KEYS", "0" if lut else str(1 << 62))
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


@pytest.mark.parametrize("mode", [0, 1])
def test_large_repair_by_groups(oracle_mod, mode):   # mode 0 runs the filtered search at radii 5, 6
    """Full-size large space in the bench's launch configuration (the scan over 695,228,960 keys
    runs with the distance tables): no constraint spans the two parameter groups, so the Hamming
    distance splits into the groups' distances and the nearest key, ties to the smallest key, is
    the nearest group-A key above the nearest group-B key.  The oracle repairs each group over its
    own valid keys."""
    from paper_2606_28372_b300 import catune as ct
    sd, sa, sb = W.large_space(), W.large_group_a(), W.large_group_b()
    sp = ct.Space.from_def(sd)
    sp.build()
    osp, oa, ob = (oracle_mod.from_def(x) for x in (sd, sa, sb))
    ka, kb = oracle_mod.valid_keys(oa), oracle_mod.valid_keys(ob)
    bits_b = int(sum(max(0, int(r - 1).bit_length()) for r in sb.n_values))
    keys = sp.keys()
    base = sp.unpack(from_dev_u64(keys[torch.from_numpy(W.random_ranks(695_228_960, 40, seed=12)).cuda()]))
    tup = np.concatenate([W.uniform_tuples(sd, 88 if mode == 0 else 24, seed=13), W.perturbed_tuples(sd, base, seed=13)])
    cand = oracle_mod.pack(osp, tup)
    sp.set_repair_mode(mode, 0)
    out = torch.empty(len(cand), dtype=torch.int64, device="cuda")
    dist = torch.empty(len(cand), dtype=torch.uint8, device="cuda")
    sp.repair(to_dev_u64(cand), out, dist)
    sp.set_repair_mode(0, 0)
    na = len(sa.n_values)
    ra, da = oracle_mod.repair(oa, ka, oracle_mod.pack(oa, tup[:, :na]))
    rb, db = oracle_mod.repair(ob, kb, oracle_mod.pack(ob, tup[:, na:]))
    want = (ra.astype(np.uint64) << np.uint64(bits_b)) | rb.astype(np.uint64)
    assert np.array_equal(from_dev_u64(out), want)
    assert np.array_equal(dist.cpu().numpy(), (da.astype(np.int64) + db).astype(np.uint8))


@pytest.mark.parametrize("path", ["near", "point", "filtered"])
def test_ball_search_spaces(oracle_mod, scan_spaces, path, monkeypatch):
    """Ball search up to radius 3 on spaces with single-value parameters, keys wider than 32 bits
    and a 300-value parameter (not filtered: more than 64 values), by each path."""
    _ball_path(path, monkeypatch)
    for sd, osp, okeys, sp in scan_spaces:
        cand = oracle_mod.pack(osp, W.uniform_tuples(sd, 96, seed=7))
        sp.set_repair_mode(2, 3)
        out = torch.empty(len(cand), dtype=torch.int64, device="cuda")
        dist = torch.empty(len(cand), dtype=torch.uint8, device="cuda")
        sp.repair(to_dev_u64(cand), out, dist)
        sp.set_repair_mode(0, 0)
        eo, ed = oracle_mod.repair(osp, okeys, cand)
        assert np.array_equal(from_dev_u64(out), eo), sd.name
        assert np.array_equal(dist.cpu().numpy(), ed), sd.name
