"""ct_repair_noalloc — the repair entry point for callers that must not allocate device memory
(an application that owns all device memory through its own allocator, or a latency-sensitive
loop that cannot afford cudaFree's device-wide synchronisation).  It must return exactly what
ct_repair returns, on consecutive calls that share its fixed scratch array.

This file is named to be collected last, so a run that stops at the first failure has already
run every other test."""
import numpy as np
import pytest
import torch

from paper_2606_28372_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(O, osp, okeys, sd, seed, count):
    base = O.unpack(osp, okeys[W.random_ranks(len(okeys), count // 2, seed)])
    c = np.concatenate([O.pack(osp, W.uniform_tuples(sd, count - count // 2, seed)),
                        O.pack(osp, W.perturbed_tuples(sd, base, seed))])
    return torch.from_numpy(c.view(np.int64)).cuda()


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_noalloc_matches_repair_on_consecutive_calls(oracle_mod, name):
    from paper_2606_28372_b300 import catune as ct
    sd = W.SPACES[name]()
    osp = oracle_mod.from_def(sd)
    okeys = oracle_mod.valid_keys(osp)
    sp = ct.Space.from_def(sd)
    sp.build()
    # two calls in a row, different sizes: the second must not see the first one's leftovers
    for seed, count in ((1, 3000), (2, 777)):
        cand = _batch(oracle_mod, osp, okeys, sd, seed, count)
        ref_out = torch.empty_like(cand)
        ref_dist = torch.empty(count, dtype=torch.uint8, device="cuda")
        sp.repair(cand, ref_out, ref_dist)
        out = torch.full_like(cand, -1)
        dist = torch.full((count,), 77, dtype=torch.uint8, device="cuda")
        sp.repair_noalloc(cand, out, dist)
        torch.cuda.synchronize()
        assert torch.equal(out, ref_out)
        assert torch.equal(dist, ref_dist)


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
