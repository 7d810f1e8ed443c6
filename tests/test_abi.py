"""The C-ABI library loads and exports every declared symbol; host-side lowering works on CPU."""
import os
import re

import numpy as np
import pytest

from paper_2606_28372_b300 import build as B
from paper_2606_28372_b300 import catune as ct
from paper_2606_28372_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "catune.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ct_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    B.build()
    L = ct.lib()
    syms = declared_symbols()
    assert len(syms) >= 25
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_layout_matches_oracle(oracle_mod):
    for name in ("tiny", "medium", "large"):
        sd = W.SPACES[name]()
        sp = ct.Space.from_def(sd)
        inf = sp.info()
        w, o, bits = oracle_mod.key_layout(oracle_mod.from_def(sd))
        assert inf.key_bits == bits
        assert list(inf.width[: inf.n_params]) == list(w)
        assert list(inf.offset[: inf.n_params]) == list(o)
        assert inf.cartesian == sd.cartesian_size and not inf.built
        idx = W.uniform_tuples(sd, 100, seed=1)
        k = sp.pack(idx)
        assert np.array_equal(k, oracle_mod.pack(oracle_mod.from_def(sd), idx))
        assert np.array_equal(sp.unpack(k), idx)


def test_define_space_errors():
    with pytest.raises(ct.CatuneError) as e:
        ct.Space(["a"] * 33, [[1, 2]] * 33, [])
    assert e.value.status == ct.CT_ERR_LIMIT
    with pytest.raises(ct.CatuneError) as e:      # 9 params x 256 values = 72 key bits
        ct.Space([f"p{i}" for i in range(9)], [list(range(256))] * 9, [])
    assert e.value.status == ct.CT_ERR_KEY_OVERFLOW
    with pytest.raises(ValueError):
        ct.Space(["a", "b"], [[1, 2], [3]], ["c > 1"])
    with pytest.raises(ct.CatuneError) as e:
        ct.Space(["a"], [[]], [])
    assert e.value.status == ct.CT_ERR_INVALID_ARG
    sp = ct.Space(["a", "b"], [[1, 2], [3, 4, 5]], ["a < b"])
    with pytest.raises(ct.CatuneError) as e:
        sp.pack([[0, 3]])
    assert e.value.status == ct.CT_ERR_INVALID_ARG


def test_postfix_program_shape():
    prog, n = ct.compile_constraints(["x", "y"], ["1 <= x*y < 9", "not (x//y == 2) or max(x, y) % 3 != 0"])
    ops = [prog[i].op for i in range(n)]
    assert ops.count(ct.OP["END"]) == 2
    # stack discipline: every program leaves exactly one value
    depth = 0
    for op in ops:
        if op in (ct.OP["PARAM"], ct.OP["CONST"]):
            depth += 1
        elif op in (ct.OP["NEG"], ct.OP["NOT"]):
            pass
        elif op == ct.OP["END"]:
            assert depth == 1
            depth = 0
        else:
            depth -= 1
