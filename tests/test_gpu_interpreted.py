"""GPU parity with every constraint interpreted per point (no truth-mask tables)."""
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

SCRIPT = r'''
import sys, numpy as np, torch
sys.path.insert(0, ".")
from oracle import oracle as O
from paper_2606_28372_b300 import workloads as W, catune as ct
from tests.helpers import from_dev_u64, to_dev_u64
for name in ("tiny", "medium"):
    sd = W.SPACES[name]()
    osp = O.from_def(sd); ok = O.valid_keys(osp)
    sp = ct.Space.from_def(sd)
    assert sp.build() == len(ok)
    assert np.array_equal(from_dev_u64(sp.keys()), ok)
    c = O.pack(osp, W.uniform_tuples(sd, 200, seed=1))
    out = torch.empty(200, dtype=torch.int64, device="cuda")
    sp.set_repair_mode(2, 2)
    sp.repair(to_dev_u64(c), out)
    assert np.array_equal(from_dev_u64(out), O.repair(osp, ok, c)[0])
print("OK")
'''


@pytest.mark.parametrize("knob", [("CATUNE_TABLE_WORDS", "0"), ("CATUNE_NO_PATTERNS", "1")])
def test_interpreted_constraints(oracle_mod, knob):
    """Both fallback build paths: every constraint interpreted per point, and truth-mask tables
    expanded per (parent, word) without per-signature patterns."""
    import os
    env = dict(os.environ)
    env[knob[0]] = knob[1]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout + r.stderr
