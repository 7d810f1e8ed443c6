"""GPU parity: the valid space built by the CUDA path equals the oracle's, key for key."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import Pair, from_dev_u64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tiny", "medium", "large_a", "large_b"])
def test_build_equals_oracle(oracle_mod, name):
    p = Pair(W.SPACES[name](), oracle_mod, table=None)
    assert p.nv == len(p.okeys)
    assert np.array_equal(p.gkeys(), p.okeys)


@pytest.mark.parametrize("s", [0, 7, 13, 22, 31])
def test_batched_spaces_equal_oracle(oracle_mod, s):
    p = Pair(W.batched_space(s), oracle_mod, table=None)
    assert np.array_equal(p.gkeys(), p.okeys)


@pytest.mark.parametrize("name", ["tiny", "medium", "large_a"])
def test_rebuild_from_previous_sizes(oracle_mod, name, monkeypatch):
    """A rebuild launches every level from the previous build's level sizes and writes the same
    keys.  With the last level's size hint one too small, that level's emit writes nothing, the
    end-of-build check fails and the level-by-level build writes the keys again; one too large
    does not fit the key buffer, so the rebuild goes level by level from the start.  The keys
    are zeroed before each rebuild, so each rebuild must write all of them itself."""
    p = Pair(W.SPACES[name](), oracle_mod, table=None)
    assert not p.sp.build_stats()["hinted"]
    first = p.sp.build_stats()["children"]

    def rebuild():
        p.sp.keys().fill_(0)
        torch.cuda.synchronize()
        assert p.sp.build() == len(p.okeys)
        st = p.sp.build_stats()
        assert st["children"] == first
        assert np.array_equal(p.gkeys(), p.okeys)
        return st["hinted"]

    assert rebuild()
    for skew in ("1", "-1"):
        monkeypatch.setenv("CATUNE_BUILD_HINT_SKEW", skew)
        assert not rebuild()
    monkeypatch.delenv("CATUNE_BUILD_HINT_SKEW")
    monkeypatch.setenv("CATUNE_BUILD_PIPELINE", "0")
    assert not rebuild()
    monkeypatch.delenv("CATUNE_BUILD_PIPELINE")
    assert rebuild()


def test_large_full_size(oracle_mod):
    """51.6e9 Cartesian points: count = |V(A)|*|V(B)|, keys strictly increasing, and sampled
    Cartesian windows equal the oracle's brute force of the same windows."""
    import torch
    from paper_2606_28372_b300 import catune as ct
    sd = W.large_space()
    sp = ct.Space.from_def(sd)
    nv = sp.build()
    assert nv == 695_228_960
    keys = sp.keys()
    # strictly increasing over the whole array (as unsigned: keys < 2^40, so signed compare is fine)
    assert bool((keys[1:] > keys[:-1]).all())
    osp = oracle_mod.from_def(sd)
    cart = sd.cartesian_size
    for c0 in [0, 7_777_777_777, 25_000_000_000, cart - 500_000]:
        c1 = min(cart, c0 + 500_000)
        exp = oracle_mod.enumerate_range(osp, c0, c1)
        idx0 = np.zeros(16, np.int64)
        t = c0
        r = sd.n_values
        for k in range(15, -1, -1):
            idx0[k] = t % r[k]
            t //= r[k]
        lo_key = int(oracle_mod.pack(osp, idx0[None])[0])
        lo = int(torch.searchsorted(keys, torch.tensor([lo_key], device="cuda")).item())
        got = from_dev_u64(keys[lo: lo + len(exp)])
        assert np.array_equal(got, exp)
        if lo + len(exp) < nv and c1 < cart:   # the next key lies beyond the window
            idx1 = np.zeros(16, np.int64)
            t = c1
            for k in range(15, -1, -1):
                idx1[k] = t % r[k]
                t //= r[k]
            hi_key = int(oracle_mod.pack(osp, idx1[None])[0])
            assert int(keys[lo + len(exp)].item()) >= hi_key
    del keys


def _large_expected_on_device(oracle_mod):
    """All 695,228,960 keys of the large space from the oracle: it is group A x group B with no
    constraint across them and A's parameters in the high bits, so its sorted keys are
    (key_A << bits_B) | key_B over the oracle's valid keys of each group, A outer."""
    ka = oracle_mod.valid_keys(oracle_mod.from_def(W.large_group_a()))
    kb = oracle_mod.valid_keys(oracle_mod.from_def(W.large_group_b()))
    osp = oracle_mod.from_def(W.large_space())
    unit = np.zeros((1, 16), np.int64)
    unit[0, 7] = 1                      # index 1 in A's lowest parameter: the key 1 << bits_B
    bits_b = int(oracle_mod.pack(osp, unit)[0]).bit_length() - 1
    a = torch.from_numpy(ka.astype(np.int64)).cuda()
    b = torch.from_numpy(kb.astype(np.int64)).cuda()
    return ((a[:, None] << bits_b) | b[None, :]).reshape(-1)


def test_large_key_for_key(oracle_mod):
    """The large space's first build and a rebuild into a zeroed key buffer (levels launched from
    the first build's sizes) both equal the oracle's keys, every one of the 695,228,960."""
    from paper_2606_28372_b300 import catune as ct
    expected = _large_expected_on_device(oracle_mod)
    assert expected.numel() == 695_228_960
    sp = ct.Space.from_def(W.large_space())
    assert sp.build() == expected.numel()
    assert not sp.build_stats()["hinted"]
    assert torch.equal(sp.keys(), expected)
    sp.keys().fill_(0)
    torch.cuda.synchronize()
    assert sp.build() == expected.numel()
    assert sp.build_stats()["hinted"]
    assert torch.equal(sp.keys(), expected)
    del expected


def test_edge_spaces(oracle_mod):
    from paper_2606_28372_b300 import catune as ct
    cases = [
        (["a", "b", "c"], [[1, 2, 3], [5, 6], [7, 8, 9, 10, 11]], []),                      # no constraints
        (["a", "b"], [[4], [1, 2, 3]], ["a % b == 0"]),                                      # single-value param
        (["a", "b"], [[-7, -1, 0, 3, 7], [-2, 0, 2, 3]], ["b == 0 or a // b >= 1", "not (a % b == 1)"]),
        (["x"], list([list(range(4096))]), ["x % 7 == 3"]),                                  # one full block
        ([f"p{i}" for i in range(12)], [[0, 1, 2]] * 12, ["p0 + p1 + p2 + p3 + p4 + p5 + p6 + p7 + p8 + p9 + p10 + p11 == 12"]),
        (["a", "b", "c"], [[1, 2], [3, 4, 5], [6]], ["1 == 1", "a < b"]),                     # constant constraint
    ]
    for names, vals, cons in cases:
        osp = oracle_mod.make_space(names, vals, cons)
        exp = oracle_mod.valid_keys(osp)
        sp = ct.Space(names, vals, cons)
        nv = sp.build(allow_empty=True)
        assert nv == len(exp), cons
        if nv:
            assert np.array_equal(from_dev_u64(sp.keys()), exp), cons


def test_empty_space_status(oracle_mod):
    from paper_2606_28372_b300 import catune as ct
    sp = ct.Space(["a", "b"], [[1, 2], [3, 4]], ["a > b"])
    with pytest.raises(ct.CatuneError) as e:
        sp.build()
    assert e.value.status == ct.CT_ERR_EMPTY_SPACE
    assert sp.info().n_valid == 0 and sp.info().built


def test_unpack_on_the_device(oracle_mod):
    """ct_unpack_keys_device against the oracle's unpacking, and the device form of the smooth
    table against the host form with the noise switched off (same bowl)."""
    from paper_2606_28372_b300 import catune as ct
    sd = W.medium_space()
    osp = oracle_mod.from_def(sd)
    ok = oracle_mod.valid_keys(osp)
    sp = ct.Space.from_def(sd)
    sp.build()
    keys = sp.keys()
    idx = torch.empty((keys.numel(), len(sd.params)), dtype=torch.int32, device="cuda")
    sp.unpack_device(keys, idx)
    exp = oracle_mod.unpack(osp, ok)
    assert np.array_equal(idx.cpu().numpy(), exp)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    dev_t = W.smooth_table_device(sd, idx, seed=3, noise=0.0, generator=g).cpu().numpy()
    host_t = W.smooth_table(sd, exp, seed=3, noise=0.0)
    assert np.allclose(dev_t, host_t, rtol=1e-6, atol=0)
