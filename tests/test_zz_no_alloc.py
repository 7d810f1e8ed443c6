"""ct_repair_noalloc — the repair entry point for callers that must not allocate device memory
(an application that owns all device memory through its own allocator, or a latency-sensitive
loop that cannot afford an allocation or cudaFree's device-wide synchronisation).  It must return
exactly what the oracle's repair returns, and what ct_repair returns, on consecutive calls that
share its fixed scratch array, including the first repair call on a freshly built space and a
batch that fills the array, and it must take no device block.

This file is named to be collected last, so a run that stops at the first failure has already
run every other test."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W
from tests.helpers import from_dev_u64, to_dev_u64

pytestmark = pytest.mark.gpu


def _batch(O, osp, okeys, sd, seed, count):
    base = O.unpack(osp, okeys[W.random_ranks(len(okeys), count // 2, seed)])
    return np.concatenate([O.pack(osp, W.uniform_tuples(sd, count - count // 2, seed)),
                           O.pack(osp, W.perturbed_tuples(sd, base, seed))])


def _noalloc(ct, sp, cand_dev):
    """One ct_repair_noalloc call into freshly filled outputs; the library's block count and
    torch's allocated bytes must not move across it."""
    n = cand_dev.numel()
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    dist = torch.full((n,), 77, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    blocks, held = ct.alloc_count(), torch.cuda.memory_allocated()
    sp.repair_noalloc(cand_dev, out, dist)
    torch.cuda.synchronize()
    assert ct.alloc_count() == blocks and torch.cuda.memory_allocated() == held
    return out, dist


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_noalloc_equals_oracle_on_consecutive_calls(oracle_mod, name):
    from paper_2606_28372_b300 import catune as ct
    sd = W.SPACES[name]()
    osp = oracle_mod.from_def(sd)
    okeys = oracle_mod.valid_keys(osp)
    sp = ct.Space.from_def(sd)
    sp.build()
    # the first repair of this space goes through the fixed scratch; then two more calls of
    # other sizes, which must not see the earlier calls' leftovers
    for i, (seed, count) in enumerate(((1, 3000), (2, 777), (3, 2048))):
        cand = _batch(oracle_mod, osp, okeys, sd, seed, count)
        cd = to_dev_u64(cand)
        out, dist = _noalloc(ct, sp, cd)
        eo, ed = oracle_mod.repair(osp, okeys, cand)
        assert np.array_equal(from_dev_u64(out), eo)
        assert np.array_equal(dist.cpu().numpy(), ed)
        if i:
            ref_out = torch.empty_like(cd)
            ref_dist = torch.empty(count, dtype=torch.uint8, device="cuda")
            sp.repair(cd, ref_out, ref_dist)
            assert torch.equal(out, ref_out) and torch.equal(dist, ref_dist)


def test_noalloc_full_batch(oracle_mod):
    """Exactly CT_REPAIR_NOALLOC_MAX candidates (every slot of the fixed arrays in use) on a
    25,895-configuration space, twice in a row, against the oracle."""
    from paper_2606_28372_b300 import catune as ct
    sd = W.large_group_a()
    osp = oracle_mod.from_def(sd)
    okeys = oracle_mod.valid_keys(osp)
    sp = ct.Space.from_def(sd)
    sp.build()
    for seed in (5, 6):
        cand = _batch(oracle_mod, osp, okeys, sd, seed, ct.REPAIR_NOALLOC_MAX)
        out, dist = _noalloc(ct, sp, to_dev_u64(cand))
        eo, ed = oracle_mod.repair(osp, okeys, cand)
        assert np.array_equal(from_dev_u64(out), eo)
        assert np.array_equal(dist.cpu().numpy(), ed)


def test_noalloc_large_by_groups(oracle_mod):
    """The full large space (695,228,960 keys): filtered ball search at the larger radii and the
    distance-table scan run through the fixed scratch.  No constraint spans the two parameter
    groups, so the nearest key is the nearest group-A key above the nearest group-B key, and the
    oracle repairs each group over its own valid keys."""
    from paper_2606_28372_b300 import catune as ct
    sd, sa, sb = W.large_space(), W.large_group_a(), W.large_group_b()
    sp = ct.Space.from_def(sd)
    sp.build()
    osp, oa, ob = (oracle_mod.from_def(x) for x in (sd, sa, sb))
    ka, kb = oracle_mod.valid_keys(oa), oracle_mod.valid_keys(ob)
    unit = np.zeros((1, 16), np.int64)
    unit[0, 7] = 1
    bits_b = int(oracle_mod.pack(osp, unit)[0]).bit_length() - 1
    base = sp.unpack(from_dev_u64(sp.keys()[torch.from_numpy(W.random_ranks(695_228_960, 40, seed=22)).cuda()]))
    tup = np.concatenate([W.uniform_tuples(sd, 88, seed=23), W.perturbed_tuples(sd, base, seed=23)])
    out, dist = _noalloc(ct, sp, to_dev_u64(oracle_mod.pack(osp, tup)))
    na = len(sa.n_values)
    ra, da = oracle_mod.repair(oa, ka, oracle_mod.pack(oa, tup[:, :na]))
    rb, db = oracle_mod.repair(ob, kb, oracle_mod.pack(ob, tup[:, na:]))
    assert np.array_equal(from_dev_u64(out), (ra.astype(np.uint64) << np.uint64(bits_b)) | rb.astype(np.uint64))
    assert np.array_equal(dist.cpu().numpy(), (da.astype(np.int64) + db).astype(np.uint8))
    assert (dist.cpu().numpy() >= 5).any()   # some candidates needed the filtered radii or the scan


def test_noalloc_rejects_oversized_batch(oracle_mod):
    from paper_2606_28372_b300 import catune as ct
    sp = ct.Space.from_def(W.tiny_space())
    sp.build()
    n = ct.REPAIR_NOALLOC_MAX + 1
    cand = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.empty_like(cand)
    with pytest.raises(ct.CatuneError) as e:
        sp.repair_noalloc(cand, out)
    assert e.value.status == ct.CT_ERR_LIMIT
